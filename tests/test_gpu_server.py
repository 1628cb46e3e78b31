"""Serving loop (hsma_server_*): continuous batching of Monte Carlo move/energy requests.

Each chain's results in the mix must equal replaying that chain's requests alone on a single
handle (within the FP32 tolerance), the committed positions must follow the accepted moves,
and admission by device footprint must hold back chains that do not fit until memory frees up.
"""
import numpy as np
import pytest

import oracle
from paper_1907_01724_gb300 import api, inputs, server

pytestmark = pytest.mark.gpu


def small_workload(count=4, n_lo=150, n_hi=1500, seed=0):
    return inputs.serving_workload(count=count, n_lo=n_lo, n_hi=n_hi, M=400, p=12, seed_offset=seed)


def replay_alone(chain, reqs_of_chain):
    """The same requests of one chain, in order, on a single handle."""
    prm = api.hsma_default_params(p=chain.p, M=chain.M, tau=chain.tau)
    h = api.hsma_create(chain.a, chain.eps1, chain.eps2, chain.kappa, prm)
    api.hsma_build_sources(h, chain.xyz, chain.q)
    out = []
    for r in reqs_of_chain:
        if r["kind"] == server.REQ_DELTA:
            out.append(api.hsma_delta_energy(h, int(r["k"]), r["x"]))
            if r["accept"]:
                api.hsma_apply_move(h, int(r["k"]), r["x"])
        else:
            out.append(api.hsma_energy(h)[0])
    return np.array(out), h


@pytest.mark.parametrize("rate", [None, 3000.0])
def test_results_same_alone_and_in_the_mix(rate):
    wl = small_workload()
    reqs, final_pos = server.make_trace(wl, 300, rate)
    srv = server.Server(wl.chains, max_batch=8, energy_slots=2)
    assert srv.hsma_server_load() == len(wl.chains)
    res = srv.hsma_server_run(reqs)
    assert np.all(res["status"] == 0)
    assert np.all(res["t_done"] >= res["t_arrival"])
    for c, chain in enumerate(wl.chains):
        mine = reqs["chain"] == c
        alone, h = replay_alone(chain, reqs[mine])
        mixed = res["value"][mine]
        # energy-scale tolerance: 1e-6 of the chain's energy terms
        e0, _ = api.hsma_energy(h)
        phi = api.hsma_potential(h)
        scale = 0.5 * np.sum(np.abs(chain.q * phi)) + abs(e0)
        assert np.max(np.abs(mixed - alone)) <= 1e-6 * scale, c
        assert np.array_equal(srv.hsma_server_positions(c), final_pos[c])


def test_final_energies_match_oracle():
    wl = small_workload(count=3, seed=5)
    reqs, final_pos = server.make_trace(wl, 120, None)
    # end every chain's stream with an energy request
    tail = np.zeros(len(wl.chains), dtype=server.REQUEST)
    for c in range(len(wl.chains)):
        tail[c]["t_arrival"] = 0.0
        tail[c]["chain"] = c
        tail[c]["kind"] = server.REQ_ENERGY
        tail[c]["id"] = 1000 + c
    srv = server.Server(wl.chains, max_batch=4, energy_slots=3)
    srv.hsma_server_load()
    res = srv.hsma_server_run(np.concatenate([reqs, tail]))
    for c, chain in enumerate(wl.chains):
        P = oracle.make_params(a=chain.a, eps1=chain.eps1, eps2=chain.eps2, kappa=chain.kappa, p=chain.p, M=chain.M)
        ref = oracle.hsma(P, final_pos[c], chain.q)
        e = res["value"][len(reqs) + c]
        scale = max(abs(ref["E_total"]), 0.5 * np.sum(np.abs(chain.q * ref["phi"])))
        assert abs(e - ref["E_total"]) <= 1e-6 * scale, (c, e, ref["E_total"], scale)


def test_admission_by_footprint_and_release():
    wl = small_workload(count=3, n_lo=800, n_hi=900, seed=9)
    # a budget that fits two of the three chains (footprint of a chain = its single-handle workspace)
    sizes = []
    for ch in wl.chains:
        h = api.hsma_create(ch.a, ch.eps1, ch.eps2, ch.kappa, api.hsma_default_params(p=ch.p, M=ch.M))
        sizes.append(api.hsma_workspace_size(h, ch.n))
    budget = int(sizes[0] + sizes[1] + 0.5 * sizes[2])
    srv = server.Server(wl.chains, hbm_budget=budget, max_batch=4)
    assert srv.hsma_server_load() == 2
    reqs = np.zeros(3, dtype=server.REQUEST)
    for c in range(3):
        reqs[c]["chain"] = c
        reqs[c]["kind"] = server.REQ_ENERGY
        reqs[c]["id"] = c
    res = srv.hsma_server_run(reqs)
    assert list(res["status"]) == [0, 0, -7]
    # closing chain 0 frees room: chain 2 is admitted and answered
    assert srv.hsma_server_close_chain(0) == 2
    res = srv.hsma_server_run(reqs)
    assert list(res["status"]) == [-7, 0, 0]


def test_invalid_requests_are_answered_not_run():
    wl = small_workload(count=2, seed=3)
    srv = server.Server(wl.chains, max_batch=4)
    srv.hsma_server_load()
    reqs = np.zeros(2, dtype=server.REQUEST)
    reqs[0]["chain"] = 0
    reqs[0]["kind"] = server.REQ_DELTA
    reqs[0]["k"] = 0
    reqs[0]["x"] = [0.0, 0.0, 10.0]
    reqs[1]["chain"] = 7
    res = srv.hsma_server_run(reqs)
    assert res["status"][0] == -2 and res["status"][1] == -1
