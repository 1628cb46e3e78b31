"""Batched evaluation of many independent cavities through the C ABI (hsma_batch_*).

Each system of a batch must match the oracle at the path's tolerance, and be bitwise identical
to the same system evaluated alone with the same pair-sum tile configuration.
"""
import numpy as np
import pytest

import oracle
from paper_1907_01724_gb300 import api, batch, inputs

pytestmark = pytest.mark.gpu

TOL = {api.HSMA_FP32: 1e-6, api.HSMA_FP64: 1e-12}


def mixed_systems(seed=3, sizes=(0, 1, 7, 100, 333, 1000, 2048, 3001)):
    rng = np.random.default_rng(seed)
    out = []
    for i, n in enumerate(sizes):
        a = float(rng.uniform(0.8, 1.5))
        ka = float(rng.uniform(0.5, 3.0))
        eps1 = 1.0 if i % 2 else 78.5
        out.append(inputs.System(a, eps1, 78.5, ka / a, 12, 400, inputs.uniform_ball(rng, n, a),
                                 inputs.neutral_charges(rng, n) if n > 1 else np.ones(n)))
    return out


def oracle_of(s):
    P = oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau)
    return oracle.hsma(P, s.xyz, s.q)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_batch_matches_oracle_per_system(prec):
    systems = mixed_systems()
    b = batch.from_systems(systems, precision=prec)
    n, xyz, q = batch.concat(systems)
    b.hsma_batch_build_sources(n, xyz, q)
    phi = b.hsma_batch_potential()
    et, er = b.hsma_batch_energy()
    off = 0
    for s, e_t, e_r in zip(systems, et, er):
        p = phi[off:off + s.n]
        off += s.n
        if s.n == 0:
            assert e_t == 0.0 and e_r == 0.0
            continue
        ref = oracle_of(s)
        assert np.linalg.norm(p - ref["phi"]) / np.linalg.norm(ref["phi"]) <= TOL[prec]
        scale = max(abs(ref["E_total"]), 0.5 * np.sum(np.abs(s.q * ref["phi"])))
        assert abs(e_t - ref["E_total"]) <= TOL[prec] * scale


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_batch_equals_alone(prec):
    """Each system of a batch matches the same system evaluated alone, and a batch is deterministic
    run to run.  The two evaluations split the sums differently (item sizes follow each system's
    share of the work), so they agree to the rounding bound of the path (1e-6 norm-wise on the
    FP32 path, the bound each of them meets against the oracle), not bitwise."""
    systems = mixed_systems(seed=9, sizes=(5, 640, 1500, 77))
    b = batch.from_systems(systems, precision=prec)
    n, xyz, q = batch.concat(systems)
    b.hsma_batch_build_sources(n, xyz, q)
    phi = b.hsma_batch_potential()
    et, _ = b.hsma_batch_energy()
    b.hsma_batch_build_sources(n, xyz, q)
    assert np.array_equal(phi, b.hsma_batch_potential())
    tol = {api.HSMA_FP32: 1e-6, api.HSMA_FP64: 1e-14}[prec]
    off = 0
    for i, s in enumerate(systems):
        alone = api.solve(s, precision=prec)
        p = phi[off:off + s.n]
        assert np.linalg.norm(alone.phi - p) <= tol * np.linalg.norm(alone.phi), i
        scale = 0.5 * np.sum(np.abs(s.q * alone.phi)) + abs(alone.E_total)
        assert abs(alone.E_total - et[i]) <= tol * scale
        off += s.n


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_batched_moves_match_single_handles(prec):
    systems = mixed_systems(seed=21, sizes=(50, 400, 900))
    b = batch.from_systems(systems, precision=prec, max_requests=8)
    n, xyz, q = batch.concat(systems)
    b.hsma_batch_build_sources(n, xyz, q)
    rng = np.random.default_rng(4)
    sys_idx, ks, xs = [], [], []
    for r in range(6):
        si = r % len(systems)
        s = systems[si]
        k = int(rng.integers(s.n))
        x_new = s.xyz[k] * 0.9
        sys_idx.append(si)
        ks.append(k)
        xs.append(x_new)
    de = b.hsma_batch_delta_energy(sys_idx, ks, xs)
    for r in range(6):
        s = systems[sys_idx[r]]
        prm = api.hsma_default_params(p=s.p, M=s.M, precision=prec)
        h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
        api.hsma_build_sources(h, s.xyz, s.q)
        d1 = api.hsma_delta_energy(h, ks[r], xs[r])
        assert abs(d1 - de[r]) <= 1e-12 * (abs(d1) + 1.0)
    # commit one move per system, then compare with the oracle on the moved configurations
    b.hsma_batch_apply_moves(sys_idx[:3], ks[:3], xs[:3])
    et, _ = b.hsma_batch_energy()
    for r in range(3):
        s = systems[sys_idx[r]]
        xyz2 = s.xyz.copy()
        xyz2[ks[r]] = xs[r]
        ref = oracle_of(inputs.System(s.a, s.eps1, s.eps2, s.kappa, s.p, s.M, xyz2, s.q))
        scale = max(abs(ref["E_total"]), 0.5 * np.sum(np.abs(s.q * ref["phi"])))
        assert abs(et[sys_idx[r]] - ref["E_total"]) <= TOL[prec] * scale


def test_two_moves_of_one_system_rejected():
    systems = mixed_systems(seed=2, sizes=(20, 30))
    b = batch.from_systems(systems, max_requests=4)
    n, xyz, q = batch.concat(systems)
    b.hsma_batch_build_sources(n, xyz, q)
    with pytest.raises(api.HsmaError):
        b.hsma_batch_apply_moves([0, 0], [1, 2], [systems[0].xyz[1] * 0.5, systems[0].xyz[2] * 0.5])


def test_autotune_picks_a_valid_config_and_stays_accurate():
    systems = mixed_systems(seed=5, sizes=(1000, 2000, 300))
    b = batch.from_systems(systems)
    n, xyz, q = batch.concat(systems)
    b.hsma_batch_build_sources(n, xyz, q)
    cfg, ms = b.hsma_batch_autotune(3)
    assert 0 <= cfg < len(batch.pair_configs()) and ms > 0
    phi = b.hsma_batch_potential()
    off = 0
    for s in systems:
        ref = oracle_of(s)
        assert np.linalg.norm(phi[off:off + s.n] - ref["phi"]) / np.linalg.norm(ref["phi"]) <= 1e-6
        off += s.n


@pytest.mark.parametrize("nsys", [1, 3])
def test_pair_schedules_agree_bitwise(nsys):
    """The real/Kelvin pair items beside the coefficient chain (schedules 1 and 2, which differ in
    the side launch's grid) or after it (0): the same items from the same work lists, so
    potentials, energies and fields are bitwise equal."""
    systems = mixed_systems(seed=9, sizes=(1500, 700, 2100)[:nsys])
    n, xyz, q = batch.concat(systems)
    out = []
    for mode in (1, 2, 0):
        b = batch.from_systems(systems)
        b.hsma_batch_set_pair_schedule(mode)
        b.hsma_batch_build_sources(n, xyz, q)
        phi = b.hsma_batch_potential()
        assert b.hsma_batch_pair_schedule() == mode
        e, _ = b.hsma_batch_energy()
        b.hsma_batch_build_sources(n, xyz, q)
        E = b.hsma_batch_field()
        out.append((phi, e, E))
    for other in out[1:]:
        for a, c in zip(out[0], other):
            assert np.array_equal(a, c)


def test_pair_schedule_rejects_bad_modes():
    b = batch.from_systems(mixed_systems(seed=9, sizes=(100,)))
    for mode in (-2, 3):
        with pytest.raises(api.HsmaError):
            b.hsma_batch_set_pair_schedule(mode)


def test_large_batch_tiles_and_surface_blocks_match_oracle():
    """A batch large enough that the moment units take several 32-charge groups per row (kg > 1:
    more than ~96 units per SM) and the surface kernel four points per warp (at least four
    blocks of 32 points per SM): per-system potentials and energies against the oracle."""
    rng = np.random.default_rng(13)
    systems = []
    for i in range(52):
        n = int(rng.integers(1700, 1900)) // 2 * 2
        a = float(rng.uniform(0.8, 1.5))
        systems.append(inputs.System(a, 1.0 if i % 2 else 78.5, 78.5, float(rng.uniform(0.5, 3.0)) / a, 20, 400,
                                     inputs.uniform_ball(rng, n, a), inputs.neutral_charges(rng, n)))
    n, xyz, q = batch.concat(systems)
    b = batch.from_systems(systems)
    b.hsma_batch_build_sources(n, xyz, q)
    phi = b.hsma_batch_potential()
    et, _ = b.hsma_batch_energy()
    off = 0
    for k, s in enumerate(systems):
        ref = oracle_of(s)
        assert np.linalg.norm(phi[off:off + s.n] - ref["phi"]) / np.linalg.norm(ref["phi"]) <= 1e-6, k
        scale = max(abs(ref["E_total"]), 0.5 * np.sum(np.abs(s.q * ref["phi"])))
        assert abs(et[k] - ref["E_total"]) <= 1e-6 * scale, k
        off += s.n
