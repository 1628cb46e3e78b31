"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: potentials norm-wise, ||phi - phi_ref||_2 / ||phi_ref||_2; energies relative to
their term scale, |E - E_ref| / max(|E_ref|, 1/2 sum_i |q_i phi_ref,i|) (a neutral system's
energy can cancel far below its terms, and no evaluation of the terms can do better than
their scale).  FP32 path 1e-6, FP64 path 1e-12.
"""
import numpy as np
import pytest

import oracle
from paper_1907_01724_gb300 import api, batch, inputs
from pointwise import record_pointwise

pytestmark = pytest.mark.gpu

TOL = {api.HSMA_FP32: 1e-6, api.HSMA_FP64: 1e-12}


def oracle_ref(s, **kw):
    P = oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau, **kw)
    return oracle.hsma(P, s.xyz, s.q)


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


def check(s, prec, ref=None, tol=None, **kw):
    tol = tol if tol is not None else TOL[prec]
    ref = ref if ref is not None else oracle_ref(s, **{k: v for k, v in kw.items() if k == "coulomb_k"})
    r = api.solve(s, precision=prec, **kw)
    e_phi = rel(r.phi, ref["phi"])
    e_rf = rel(r.phi_rf, ref["phi_rf"])
    # the pointwise errors are reported beside the norm-wise ones (the pointwise relative error is
    # ill-conditioned where a potential nearly cancels, so it is recorded, not asserted)
    record_pointwise(f"{s.name or 'N%d' % s.n} {'fp32' if prec == api.HSMA_FP32 else 'fp64'}", prec, r.phi,
                     ref["phi"], e_phi)
    scale_t = max(abs(ref["E_total"]), 0.5 * np.sum(np.abs(s.q * ref["phi"])), 1e-300)
    scale_r = max(abs(ref["E_rf"]), 0.5 * np.sum(np.abs(s.q * ref["phi_rf"])), 1e-300)
    e_E = abs(r.E_total - ref["E_total"]) / scale_t
    e_Erf = abs(r.E_rf - ref["E_rf"]) / scale_r
    assert e_phi <= tol, ("phi", e_phi)
    assert e_rf <= tol, ("phi_rf", e_rf)
    assert e_E <= tol, ("E", e_E)
    assert e_Erf <= tol, ("E_rf", e_Erf)
    return r, ref


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_small_uniform_system(prec):
    check(inputs.small_system(), prec)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
@pytest.mark.parametrize("ka", [0.5, 2.0])
def test_near_interface_system(prec, ka):
    check(inputs.near_interface_system(kappa_a=ka), prec)


def test_near_interface_p30_fp32():
    check(inputs.near_interface_system(kappa_a=2.0, p=30), api.HSMA_FP32)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_primitive_full_size(prec):
    """N = 20000, eps1 = eps2 = 78.5, kappa a = 3, M = 2000, p = 30, compared at full size."""
    s = inputs.primitive_system()
    ref = oracle_ref(s)
    check(s, prec, ref=ref)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_clustered_charges_dense_cells(prec):
    """6000 charges in a ball of radius 0.06 a off the centre: a handful of the spatial order's
    16^3 cells hold hundreds of charges each, and the sort block that owns them has more charges
    than its shared memory (it sorts in the scratch buffer)."""
    rng = np.random.default_rng(4242)
    n = 6000
    xyz = inputs.uniform_ball(rng, n, 0.06) + np.array([0.31, -0.12, 0.2])
    s = inputs.System(1.0, 2.0, 80.0, 1.0, 12, 200, xyz, rng.choice([-1.0, 1.0], n))
    check(s, prec)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
@pytest.mark.parametrize("n", [1, 2, 3, 31, 517, 1029])
def test_ragged_sizes(prec, n):
    rng = np.random.default_rng(1000 + n)
    s = inputs.System(1.0, 1.0, 80.0, 1.0, 12, 200, inputs.uniform_ball(rng, n, 0.99),
                      rng.choice([-1.0, 1.0], n))
    check(s, prec)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_edge_geometries(prec):
    cases = [
        np.array([[0.0, 0.0, 0.0]]),                              # centre: image at infinity
        np.array([[0.0, 0.0, 0.999999]]),                         # touching the interface
        np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.1]]),            # centre + another
        np.array([[0.5, 0.5, 0.5], [-0.5, 0.5, -0.5], [0.0, -0.99, 0.0]]),
    ]
    for xyz in cases:
        q = np.array([1.0, -2.0, 0.5][: len(xyz)])
        s = inputs.System(1.3, 2.0, 80.0, 5.0 / 1.3, 20, 400, xyz * 1.3, q)
        check(s, prec)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_degenerate_parameters(prec):
    rng = np.random.default_rng(77)
    xyz = inputs.uniform_ball(rng, 64, 0.95)
    q = inputs.neutral_charges(rng, 64)
    # no dielectric jump and no screening: zero reaction potential
    s = inputs.System(1.0, 5.0, 5.0, 0.0, 10, 100, xyz, q)
    r, ref = check(s, prec)
    assert np.max(np.abs(r.phi_rf)) < 1e-12 * np.max(np.abs(r.phi))
    # Poisson outside (kappa = 0), p = 0, the minimum M, Gaussian units
    check(inputs.System(1.0, 1.0, 80.0, 0.0, 16, 400, xyz, q), prec)
    check(inputs.System(1.0, 1.0, 80.0, 1.0, 0, 4, xyz, q), prec)
    check(inputs.System(0.7, 1.0, 78.5, 2.0, 8, 100, xyz * 0.7, q), prec, coulomb_k=1.0)


def test_high_order_paper_parameters():
    """The paper's Sec. 4 parameters (F1 = 987, F2 = 1597) at p = 55 for a near-interface charge."""
    xyz = np.array([[0.0, 0.0, 0.95]])
    q = np.array([1.0])
    P = oracle.make_params(a=1, eps1=2, eps2=80, kappa=5, p=55, F1=987, F2=1597)
    ref = oracle.hsma(P, xyz, q)
    for prec in (api.HSMA_FP32, api.HSMA_FP64):
        prm = api.hsma_default_params(p=55, F1=987, F2=1597, precision=prec)
        h = api.hsma_create(1.0, 2.0, 80.0, 5.0, prm)
        api.hsma_build_sources(h, xyz, q)
        et, er = api.hsma_energy(h)
        assert abs(er - ref["E_rf"]) / abs(ref["E_rf"]) <= TOL[prec]


def test_empty_system():
    s = inputs.System(1.0, 1.0, 80.0, 1.0, 10, 100, np.zeros((0, 3)), np.zeros(0))
    r = api.solve(s)
    assert r.phi.shape == (0,) and r.E_total == 0.0 and r.E_rf == 0.0


def test_errors_are_reported():
    prm = api.hsma_default_params(p=8, M=100)
    h = api.hsma_create(1.0, 1.0, 80.0, 1.0, prm)
    with pytest.raises(api.HsmaError) as e:
        api.hsma_potential(h)
    assert e.value.code == -3
    api.hsma_build_sources(h, np.array([[0.0, 0.0, 1.0]]), np.array([1.0]))  # checked on the device
    with pytest.raises(api.HsmaError) as e:
        api.hsma_potential(h)
    assert e.value.code == -2
    api.hsma_build_sources(h, np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3]]), np.array([1.0, -1.0]))
    with pytest.raises(api.HsmaError) as e:
        api.hsma_potential(h)
    assert e.value.code == -8
    with pytest.raises(api.HsmaError) as e:
        api.hsma_create(-1.0, 1.0, 80.0, 1.0, prm)
    assert e.value.code == -1
    bad = api.hsma_default_params(p=8, M=7)
    with pytest.raises(api.HsmaError):
        api.hsma_create(1.0, 1.0, 80.0, 1.0, bad)


def test_device_outside_charge_detected_by_kernel():
    import torch
    prm = api.hsma_default_params(p=8, M=100)
    h = api.hsma_create(1.0, 1.0, 80.0, 1.0, prm)
    xyz = torch.tensor([[0.1, 0.0, 0.0], [0.0, 0.0, 1.5]], dtype=torch.float64, device="cuda")
    q = torch.tensor([1.0, -1.0], dtype=torch.float64, device="cuda")
    api.hsma_build_sources(h, xyz, q)
    with pytest.raises(api.HsmaError) as e:
        api.hsma_energy(h)
    assert e.value.code == -2


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_device_resident_path_matches_host_path(prec):
    import torch
    s = inputs.near_interface_system(kappa_a=0.5)
    prm = api.hsma_default_params(p=s.p, M=s.M, precision=prec)
    h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
    api.hsma_build_sources(h, s.xyz, s.q)
    phi_host = api.hsma_potential(h)
    xyz_d = torch.tensor(s.xyz, device="cuda")
    q_d = torch.tensor(s.q, device="cuda")
    api.hsma_build_sources(h, xyz_d, q_d)
    out = torch.empty(s.n, dtype=torch.float64, device="cuda")
    api.hsma_potential(h, out=out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), phi_host)


def test_results_are_deterministic():
    s = inputs.near_interface_system(kappa_a=2.0)
    a = api.solve(s)
    b = api.solve(s)
    assert np.array_equal(a.phi, b.phi) and a.E_total == b.E_total


@pytest.mark.parametrize("p", [20, 30, 55])
def test_double_float_coefficients_match_fp64(p):
    """The FP32 path evaluates the solid-harmonic moments and surface synthesis in double-float
    arithmetic (~2^-46); its correction coefficients must match the FP64 path's to 1e-12."""
    s = inputs.near_interface_system(kappa_a=2.0, n=1000)
    co = []
    for prec in (api.HSMA_FP32, api.HSMA_FP64):
        prm = api.hsma_default_params(p=p, M=2 * p * p + 2, precision=prec)
        h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
        api.hsma_build_sources(h, s.xyz, s.q)
        co.append(api.hsma_coefficients(h, p))
    assert np.linalg.norm(co[0] - co[1]) <= 1e-12 * np.linalg.norm(co[1])


def test_kernel_launch_accounting():
    s = inputs.small_system()
    prm = api.hsma_default_params(p=s.p, M=s.M)
    h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
    api.hsma_build_sources(h, s.xyz, s.q)
    api.hsma_energy(h)
    # once per layout: k_setup, k_surface_basis; build: k_order_keys, k_order_sort, k_images,
    # k_moment_prep, k_moment_units, k_coef_reduce, k_surface_mat; potentials (the build and
    # the pass in one graph; a single cavity's default schedule): k_pairs (real/Kelvin items,
    # beside the coefficient chain), k_pairs (surface items, then the real/Kelvin items left),
    # k_reduce
    assert api.hsma_kernel_launches(h) == 12
    api.hsma_set_overlap(h, False)
    api.hsma_build_sources(h, s.xyz, s.q)
    api.hsma_energy(h)
    # separate passes: the 7 build kernels, then k_pairs and k_reduce
    assert api.hsma_kernel_launches(h) == 12 + 9


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_overlapped_and_separate_passes_agree_bitwise(prec):
    s = inputs.near_interface_system(kappa_a=2.0)
    prm = api.hsma_default_params(p=s.p, M=s.M, precision=prec)
    h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
    api.hsma_build_sources(h, s.xyz, s.q)
    phi1 = api.hsma_potential(h)
    e1 = api.hsma_energy(h)
    api.hsma_set_overlap(h, False)
    api.hsma_build_sources(h, s.xyz, s.q)
    phi0 = api.hsma_potential(h)
    e0 = api.hsma_energy(h)
    api.hsma_destroy(h)
    assert np.array_equal(phi0, phi1)
    assert e0 == e1


@pytest.mark.parametrize("bad", ["nan_x", "inf_z", "inf_q", "nan_q", "on_sphere", "last_of_many"])
def test_host_inputs_checked_on_the_device(bad):
    """A charge at |x| >= a or a non-finite coordinate or charge in host inputs is found by the
    pass's first kernel and reported by the evaluation (HSMA_E_OUTSIDE = -2), single handle and
    batch, wherever it sits in the array; a corrected build then evaluates normally."""
    rng = np.random.default_rng(5)
    xyz = inputs.uniform_ball(rng, 300, 0.9)
    q = rng.choice([-1.0, 1.0], size=300)
    k = 299 if bad == "last_of_many" else 17
    if bad == "nan_x":
        xyz[k, 0] = np.nan
    elif bad == "inf_z":
        xyz[k, 2] = -np.inf
    elif bad == "inf_q":
        q[k] = np.inf
    elif bad == "nan_q":
        q[k] = np.nan
    elif bad == "on_sphere":
        xyz[k] = (0.0, 1.0, 0.0)
    else:
        xyz[k] = (0.6, 0.6, 0.6)
    prm = api.hsma_default_params(p=8, M=100)
    h = api.hsma_create(1.0, 1.0, 80.0, 1.0, prm)
    api.hsma_build_sources(h, xyz, q)
    with pytest.raises(api.HsmaError) as e:
        api.hsma_energy(h)
    assert e.value.code == -2
    xyz_ok = inputs.uniform_ball(rng, 300, 0.9)
    api.hsma_build_sources(h, xyz_ok, np.abs(q) if np.all(np.isfinite(q)) else np.ones(300))
    assert np.all(np.isfinite(api.hsma_potential(h)))
    api.hsma_destroy(h)
    good = inputs.uniform_ball(rng, 50, 0.9)
    b = batch.Batch([1.0, 1.0], [1.0, 1.0], [80.0, 80.0], [1.0, 1.0], prm)
    b.hsma_batch_build_sources([50, 300], np.concatenate([good, xyz]), np.concatenate([np.ones(50), q]))
    with pytest.raises(api.HsmaError) as e:
        b.hsma_batch_potential()
    assert e.value.code == -2
