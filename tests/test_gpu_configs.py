"""Every pair-sum tile configuration (CTA threads, targets per thread, items per slot) against the
FP64 oracle: potentials, energies and fields of a ragged batch, FP32 path (norm-wise 1e-6, as
everywhere)."""
import numpy as np
import pytest

import oracle
from paper_1907_01724_gb300 import api, batch, inputs

pytestmark = pytest.mark.gpu


def P_of(s):
    return oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(41)
    systems = [inputs.System(xyz=inputs.uniform_ball(rng, n, 1.0), q=rng.choice([-1.0, 1.0], size=n), a=1.0,
                             eps1=1.0, eps2=78.5, kappa=1.5, p=12, M=400, tau=0.1) for n in (5, 300, 1100)]
    near = inputs.near_interface_system(kappa_a=2.0)
    systems.append(inputs.System(xyz=near.xyz, q=near.q, a=near.a, eps1=near.eps1, eps2=near.eps2, kappa=near.kappa,
                                 p=12, M=400, tau=0.1))
    # several blocks with a centre charge (image at infinity: exactly at the centre, and inside the
    # centre threshold), so that the both-way Kelvin terms of centre charges are exercised
    for c in ([0.0, 0.0, 0.0], [1e-13, -2e-13, 0.0]):
        xyz = np.concatenate([inputs.uniform_ball(rng, 1299, 1.0), [c]])
        systems.append(inputs.System(xyz=xyz, q=inputs.neutral_charges(rng, 1300), a=1.0, eps1=2.0, eps2=78.5,
                                     kappa=1.0, p=12, M=400, tau=0.1))
    refs = []
    for s in systems:
        r = oracle.hsma(P_of(s), s.xyz, s.q)
        r["E"] = oracle.field(P_of(s), s.xyz, s.q)["E"]
        refs.append(r)
    return systems, refs


def _configs():
    try:
        return list(range(len(batch.pair_configs())))
    except Exception:  # library not built (collection on a machine without the extension)
        return [0]


@pytest.mark.parametrize("cfg", _configs())
def test_pair_config_matches_oracle(case, cfg):
    systems, refs = case
    n, xyz, q = batch.concat(systems)
    b = batch.from_systems(systems, precision=api.HSMA_FP32)
    b.hsma_batch_set_pair_config(cfg)
    b.hsma_batch_build_sources(n, xyz, q)
    phi = b.hsma_batch_potential()
    et, _ = b.hsma_batch_energy()
    E = b.hsma_batch_field()
    off = 0
    for k, (s, r) in enumerate(zip(systems, refs)):
        assert rel(phi[off:off + s.n], r["phi"]) <= 1e-6, (batch.pair_configs()[cfg], k)
        assert rel(E[off:off + s.n], r["E"]) <= 1e-6, (batch.pair_configs()[cfg], k)
        scale = max(abs(r["E_total"]), 0.5 * np.sum(np.abs(s.q * r["phi"])))
        assert abs(et[k] - r["E_total"]) <= 1e-6 * scale
        off += s.n
