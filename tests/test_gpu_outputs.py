"""Where a potential pass writes its results: straight into the caller's array (device output) or
pinned staging (host output) when the call runs the pass, by copies when the potentials are
already current; a later pass that asks for no output must leave earlier destinations alone."""
import numpy as np
import pytest

import oracle
from paper_1907_01724_gb300 import api, batch, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def systems():
    rng = np.random.default_rng(31)
    return [inputs.System(xyz=inputs.uniform_ball(rng, n, 1.0), q=rng.choice([-1.0, 1.0], size=n), a=1.0, eps1=1.0,
                          eps2=78.5, kappa=1.0, p=12, M=400, tau=0.1) for n in (700, 129)]


def refs(sy):
    out = []
    for s in sy:
        P = oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau)
        out.append(oracle.hsma(P, s.xyz, s.q))
    return out


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_device_and_host_outputs_alternate(prec):
    tol = 1e-6 if prec == api.HSMA_FP32 else 1e-12
    sy = systems()
    ref = refs(sy)
    n, xyz, q = batch.concat(sy)
    tot = int(n.sum())
    key = {api.HSMA_TOTAL: "phi", api.HSMA_REACTION: "phi_rf", api.HSMA_COULOMB: "phi_coul"}
    want = {w: np.concatenate([r[k] for r in ref]) for w, k in key.items()}
    b = batch.from_systems(sy, precision=prec)
    A = torch.full((tot,), -7.0, dtype=torch.float64, device="cuda")
    B = torch.full((tot,), -7.0, dtype=torch.float64, device="cuda")
    # the pass runs in this call and writes A itself
    b.hsma_batch_build_sources(n, xyz, q)
    b.hsma_batch_potential(api.HSMA_REACTION, out=A)
    torch.cuda.synchronize()
    a1 = A.cpu().numpy()
    assert rel(a1, want[api.HSMA_REACTION]) <= tol
    # potentials current: copies, into B, another quantity
    b.hsma_batch_potential(api.HSMA_COULOMB, out=B)
    torch.cuda.synchronize()
    assert rel(B.cpu().numpy(), want[api.HSMA_COULOMB]) <= tol
    # a new pass that asks for no output (energies) must not touch A or B
    A.fill_(-7.0)
    B.fill_(-7.0)
    b.hsma_batch_build_sources(n, xyz, q)
    et, _ = b.hsma_batch_energy()
    torch.cuda.synchronize()
    assert np.all(A.cpu().numpy() == -7.0) and np.all(B.cpu().numpy() == -7.0)
    for k, (s, r) in enumerate(zip(sy, ref)):
        scale = max(abs(r["E_total"]), 0.5 * np.sum(np.abs(s.q * r["phi"])))
        assert abs(et[k] - r["E_total"]) <= tol * scale
    # host output of a fresh pass, then device output of the next, then host again
    for w in (api.HSMA_TOTAL, api.HSMA_COULOMB):
        b.hsma_batch_build_sources(n, xyz, q)
        h = b.hsma_batch_potential(w)
        assert rel(h, want[w]) <= tol
        e1 = b.hsma_batch_energy()
        b.hsma_batch_build_sources(n, xyz, q)
        b.hsma_batch_potential(w, out=B)
        torch.cuda.synchronize()
        assert np.array_equal(B.cpu().numpy(), h)
        assert np.array_equal(np.asarray(b.hsma_batch_energy()), np.asarray(e1))
    assert np.all(A.cpu().numpy() == -7.0)


def test_single_handle_outputs():
    s = systems()[0]
    ref = refs([s])[0]
    prm = api.hsma_default_params(p=s.p, M=s.M, tau=s.tau)
    h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
    api.hsma_build_sources(h, s.xyz, s.q)
    out = torch.full((s.n,), -7.0, dtype=torch.float64, device="cuda")
    api.hsma_potential(h, api.HSMA_TOTAL, out=out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), ref["phi"]) <= 1e-6
    host = api.hsma_potential(h, api.HSMA_TOTAL)
    assert np.array_equal(host, out.cpu().numpy())
    out.fill_(-7.0)
    api.hsma_build_sources(h, s.xyz, s.q)
    host2 = api.hsma_potential(h, api.HSMA_REACTION)
    assert rel(host2, ref["phi_rf"]) <= 1e-6
    et, er = api.hsma_energy(h)
    assert abs(et - ref["E_total"]) <= 1e-6 * max(abs(ref["E_total"]), 0.5 * np.sum(np.abs(s.q * ref["phi"])))
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == -7.0)
    api.hsma_destroy(h)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_call_sequences_after_host_outputs(prec):
    """Builds, host and device potentials of different quantities, fields and energies in
    sequence: whatever the caller asks next gets the results of the current positions (the
    pinned staging of a host-output pass is never mistaken for a later pass's values)."""
    tol = 1e-6 if prec == api.HSMA_FP32 else 1e-12
    sy = systems()
    n, xyz, q = batch.concat(sy)
    rng = np.random.default_rng(77)
    xyz2 = xyz.copy()
    xyz2[::7] *= 0.97  # moved charges (still inside)
    sy2 = [inputs.System(xyz=xyz2[a:a + s.n], q=s.q, a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M,
                         tau=s.tau) for s, a in zip(sy, np.cumsum([0] + [s.n for s in sy])[:-1])]
    r1, r2 = refs(sy), refs(sy2)
    phi1 = np.concatenate([r["phi"] for r in r1])
    phi2 = np.concatenate([r["phi"] for r in r2])
    rf2 = np.concatenate([r["phi_rf"] for r in r2])
    b = batch.from_systems(sy, precision=prec)
    b.hsma_batch_build_sources(n, xyz, q)
    assert rel(b.hsma_batch_potential(), phi1) <= tol
    b.hsma_batch_build_sources(n, xyz2, q)
    assert rel(b.hsma_batch_potential(), phi2) <= tol
    et, _ = b.hsma_batch_energy()
    for k, (s, r) in enumerate(zip(sy2, r2)):
        scale = max(abs(r["E_total"]), 0.5 * np.sum(np.abs(s.q * r["phi"])))
        assert abs(et[k] - r["E_total"]) <= tol * scale
    # another quantity of the early pass, then a field request, then potentials again
    b.hsma_batch_build_sources(n, xyz, q)
    b.hsma_batch_build_sources(n, xyz2, q)
    assert rel(b.hsma_batch_potential(api.HSMA_REACTION), rf2) <= tol
    assert rel(b.hsma_batch_potential(), phi2) <= tol
    b.hsma_batch_build_sources(n, xyz, q)
    E = b.hsma_batch_field()
    off = 0
    for s in sy:
        P = oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau)
        assert rel(E[off:off + s.n], oracle.field(P, s.xyz, s.q)["E"]) <= tol
        off += s.n
    assert rel(b.hsma_batch_potential(), phi1) <= tol
    # energies only, after two builds
    b.hsma_batch_build_sources(n, xyz2, q)
    b.hsma_batch_build_sources(n, xyz2, q)
    et, _ = b.hsma_batch_energy()
    for k, (s, r) in enumerate(zip(sy2, r2)):
        scale = max(abs(r["E_total"]), 0.5 * np.sum(np.abs(s.q * r["phi"])))
        assert abs(et[k] - r["E_total"]) <= tol * scale


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_device_inputs_read_in_place(prec):
    """Device inputs are read by the evaluation that runs the build pass, which keeps its own
    copy: results follow the positions at that evaluation; rewriting the caller's array after it
    changes nothing the handle returns (another quantity, a field pass) until the next build; the
    autotuner, run while a build from device arrays is pending, tunes and leaves the handle on
    those inputs."""
    tol = 1e-6 if prec == api.HSMA_FP32 else 1e-12
    sy = systems()
    n, xyz, q = batch.concat(sy)
    xyz2 = xyz * 0.97
    sy2 = [inputs.System(xyz=xyz2[a:a + s.n], q=s.q, a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M,
                         tau=s.tau) for s, a in zip(sy, np.cumsum([0] + [s.n for s in sy])[:-1])]
    r1, r2 = refs(sy), refs(sy2)
    phi1 = np.concatenate([r["phi"] for r in r1])
    rf1 = np.concatenate([r["phi_rf"] for r in r1])
    phi2 = np.concatenate([r["phi"] for r in r2])
    b = batch.from_systems(sy, precision=prec)
    xyz_d = torch.tensor(xyz, device="cuda")
    q_d = torch.tensor(q, device="cuda")
    b.hsma_batch_build_sources(n, xyz_d, q_d)
    assert rel(b.hsma_batch_potential(), phi1) <= tol
    xyz_d.mul_(0.97)  # the caller rewrites its array after the evaluation
    torch.cuda.synchronize()
    assert rel(b.hsma_batch_potential(api.HSMA_REACTION), rf1) <= tol
    E = b.hsma_batch_field()
    off = 0
    for s in sy:
        P = oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau)
        assert rel(E[off:off + s.n], oracle.field(P, s.xyz, s.q)["E"]) <= tol
        off += s.n
    # the next build reads the rewritten array
    b.hsma_batch_build_sources(n, xyz_d, q_d)
    assert rel(b.hsma_batch_potential(), phi2) <= tol
    if prec == api.HSMA_FP32:
        # a pending build from device arrays, then the autotuner, then an evaluation
        xyz1_d = torch.tensor(xyz, device="cuda")
        b.hsma_batch_build_sources(n, xyz1_d, q_d)
        b.hsma_batch_autotune(1)
        assert rel(b.hsma_batch_potential(), phi1) <= tol


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_page_locked_host_buffers(prec):
    """Page-locked host inputs are read in place by the evaluation (like device inputs) and a
    page-locked output array is written by the device itself: the results equal those of the
    pageable path bitwise; rewriting the page-locked inputs after the evaluation changes nothing
    the handle returns until the next build, which reads the new values."""
    tol = 1e-6 if prec == api.HSMA_FP32 else 1e-12
    sy = systems()
    n, xyz, q = batch.concat(sy)
    tot = int(n.sum())
    r1 = refs(sy)
    phi1 = np.concatenate([r["phi"] for r in r1])
    b = batch.from_systems(sy, precision=prec)
    b.hsma_batch_build_sources(n, xyz, q)
    ref_pageable = b.hsma_batch_potential()
    e_pageable, _ = b.hsma_batch_energy()
    xyz_h = torch.tensor(xyz).pin_memory().numpy()
    q_h = torch.tensor(q).pin_memory().numpy()
    out_h = torch.full((tot,), -7.0, dtype=torch.float64).pin_memory().numpy()
    b.hsma_batch_build_sources(n, xyz_h, q_h)
    got = b.hsma_batch_potential(out=out_h)
    assert got is out_h
    assert np.array_equal(out_h, ref_pageable)
    e_pinned, _ = b.hsma_batch_energy()
    assert np.array_equal(e_pinned, e_pageable)
    assert rel(out_h, phi1) <= tol
    xyz_h *= 0.97  # the caller rewrites its page-locked inputs after the evaluation
    out_h[:] = -7.0
    b.hsma_batch_potential(out=out_h)  # the current pass: copied into the page-locked array
    assert np.array_equal(out_h, ref_pageable)
    b.hsma_batch_build_sources(n, xyz_h, q_h)
    sy2 = [inputs.System(xyz=xyz_h[a:a + s.n].copy(), q=s.q, a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p,
                         M=s.M, tau=s.tau) for s, a in zip(sy, np.cumsum([0] + [s.n for s in sy])[:-1])]
    phi2 = np.concatenate([r["phi"] for r in refs(sy2)])
    assert rel(b.hsma_batch_potential(out=out_h), phi2) <= tol
    h = api.hsma_create(1.0, 1.0, 78.5, 1.0, api.hsma_default_params(p=12, M=400, precision=prec))
    try:
        api.hsma_build_sources(h, xyz_h[:sy[0].n], q_h[:sy[0].n])
        one = torch.empty(sy[0].n, dtype=torch.float64).pin_memory().numpy()
        api.hsma_potential(h, out=one)
        assert rel(one, phi2[:sy[0].n]) <= tol
    finally:
        api.hsma_destroy(h)
