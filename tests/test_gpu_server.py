"""Serving loop (hsma_server_*): continuous batching of Monte Carlo move/energy requests.

Each chain's results in the mix must equal replaying that chain's requests alone on a single
handle (within the FP32 tolerance), the committed positions must follow the accepted moves,
and admission by device footprint must hold back chains that do not fit until memory frees up.
"""
import ctypes
import threading
import time

import numpy as np
import pytest

import oracle
from paper_1907_01724_gb300 import _native, api, inputs, server

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
    # chain 2 is not resident: its request waits until an idle chain is evicted, then is answered
    res = srv.hsma_server_run(reqs)
    assert list(res["status"]) == [0, 0, 0]
    for c, chain in enumerate(wl.chains):
        P = oracle.make_params(a=chain.a, eps1=chain.eps1, eps2=chain.eps2, kappa=chain.kappa, p=chain.p, M=chain.M)
        ref = oracle.hsma(P, chain.xyz, chain.q)
        scale = max(abs(ref["E_total"]), 0.5 * np.sum(np.abs(chain.q * ref["phi"])))
        assert abs(res["value"][c] - ref["E_total"]) <= 1e-6 * scale, c
    # a closed chain's requests are refused; the others are served
    assert srv.hsma_server_close_chain(0) == 2
    res = srv.hsma_server_run(reqs)
    assert list(res["status"]) == [-7, 0, 0]


def test_chain_larger_than_the_budget_is_refused():
    wl = small_workload(count=2, n_lo=800, n_hi=900, seed=4)
    h = api.hsma_create(wl.chains[0].a, wl.chains[0].eps1, wl.chains[0].eps2, wl.chains[0].kappa,
                        api.hsma_default_params(p=wl.chains[0].p, M=wl.chains[0].M))
    small = api.hsma_workspace_size(h, 10)
    # chain 1 gets far more charges than the budget allows
    big = inputs.System(wl.chains[1].a, wl.chains[1].eps1, wl.chains[1].eps2, wl.chains[1].kappa, wl.chains[1].p,
                        wl.chains[1].M, inputs.uniform_ball(np.random.default_rng(1), 20000, 0.99 * wl.chains[1].a),
                        inputs.neutral_charges(np.random.default_rng(2), 20000))
    chains = [inputs.System(c.a, c.eps1, c.eps2, c.kappa, c.p, c.M, c.xyz[:10], c.q[:10]) for c in wl.chains[:1]]
    srv = server.Server(chains + [big], hbm_budget=int(3 * small), max_batch=4)
    assert srv.hsma_server_load() == 1
    reqs = np.zeros(2, dtype=server.REQUEST)
    for c in range(2):
        reqs[c]["chain"] = c
        reqs[c]["kind"] = server.REQ_ENERGY
    res = srv.hsma_server_run(reqs)
    assert list(res["status"]) == [0, -7]


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


# --- the live boundary: producers submit while the loop runs ------------------------------

def _poll_all(srv, n, timeout=60.0):
    got, total = [], 0
    t_end = time.monotonic() + timeout
    while total < n and time.monotonic() < t_end:
        r = srv.hsma_server_poll(512, 0.05)
        if len(r):
            got.append(r)
            total += len(r)
    return np.concatenate(got) if got else np.zeros(0, dtype=server.RESULT)


def test_live_producer_thread_results_equal_alone():
    """A producer thread submits a Poisson stream while earlier requests are on the GPU; the main
    thread polls.  Every chain's answers equal replaying its requests alone on a single handle."""
    wl = small_workload(seed=21)
    reqs, final_pos = server.make_trace(wl, 400, 4000.0)
    srv = server.Server(wl.chains, max_batch=8, energy_slots=2)
    srv.hsma_server_load()
    srv.hsma_server_start()
    tickets = {}

    def producer():
        t0 = time.monotonic()
        for i, r in enumerate(reqs):
            dt = r["t_arrival"] - (time.monotonic() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets[srv.hsma_server_submit(r)] = i

    th = threading.Thread(target=producer)
    th.start()
    res = _poll_all(srv, len(reqs))
    th.join()
    srv.hsma_server_stop(drain=True)
    assert len(res) == len(reqs)
    assert np.all(res["status"] == 0)
    # in flight together: some request was submitted before an earlier one was answered
    order = np.argsort(res["ticket"])
    assert np.any(res["t_arrival"][order][1:] < res["t_done"][order][:-1])
    by_index = np.zeros(len(reqs), dtype=server.RESULT)
    for r in res:
        by_index[tickets[int(r["ticket"])]] = r
    assert np.array_equal(by_index["id"], reqs["id"])
    for c, chain in enumerate(wl.chains):
        mine = reqs["chain"] == c
        alone, h = replay_alone(chain, reqs[mine])
        e0, _ = api.hsma_energy(h)
        phi = api.hsma_potential(h)
        scale = 0.5 * np.sum(np.abs(chain.q * phi)) + abs(e0)
        assert np.max(np.abs(by_index["value"][mine] - alone)) <= 1e-6 * scale, c
        assert np.array_equal(srv.hsma_server_positions(c), final_pos[c])


def test_producer_stops_midway_and_the_loop_drains():
    """The producer thread dies part-way through its stream (an exception on the host, no stop
    call from it); the owner stops the loop with drain, and every request that was submitted
    is answered."""
    wl = small_workload(seed=23)
    reqs, _ = server.make_trace(wl, 300, None)
    srv = server.Server(wl.chains, max_batch=8, energy_slots=2)
    srv.hsma_server_load()
    srv.hsma_server_start()
    submitted, fault = [], []

    def producer():
        try:
            for i, r in enumerate(reqs):
                if i == 120:
                    raise RuntimeError("producer fault")
                submitted.append(srv.hsma_server_submit(r))
        except RuntimeError as exc:  # the producer's thread ends here, without stopping the loop
            fault.append(exc)

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    assert len(submitted) == 120 and len(fault) == 1
    srv.hsma_server_stop(drain=True)
    res = _poll_all(srv, len(submitted), timeout=5.0)
    assert sorted(res["ticket"].tolist()) == sorted(submitted)
    assert np.all(res["status"] == 0)
    # the loop is stopped: a late submission is refused
    with pytest.raises(api.HsmaError) as e:
        srv.hsma_server_submit(reqs[130])
    assert e.value.code == -3


def test_stop_without_drain_cancels_what_has_not_started():
    wl = small_workload(count=1, n_lo=1400, n_hi=1500, seed=25)
    srv = server.Server(wl.chains, max_batch=8, energy_slots=1)
    srv.hsma_server_load()
    srv.hsma_server_start()
    reqs = np.zeros(200, dtype=server.REQUEST)
    reqs["kind"] = server.REQ_ENERGY
    reqs["id"] = np.arange(200)
    tickets = [srv.hsma_server_submit(r) for r in reqs]
    srv.hsma_server_stop(drain=False)
    res = _poll_all(srv, len(tickets), timeout=5.0)
    assert sorted(res["ticket"].tolist()) == tickets
    assert set(res["status"].tolist()) <= {0, -7}
    assert np.sum(res["status"] == -7) > 0
    # answers that completed are the chain's energy
    ok = res["status"] == 0
    if ok.any():
        assert np.allclose(res["value"][ok], res["value"][ok][0], rtol=0, atol=0)


def test_poll_deadline_and_restart():
    wl = small_workload(count=2, seed=27)
    srv = server.Server(wl.chains, max_batch=4)
    srv.hsma_server_load()
    srv.hsma_server_start()
    lib = srv.lib
    out = np.zeros(4, dtype=server.RESULT)
    cnt = ctypes.c_int()
    t0 = time.monotonic()
    rc = lib.hsma_server_poll(srv.ptr, _native.host_ptr(out), 4, 0.05, ctypes.byref(cnt))
    assert rc == server.HSMA_E_TIMEOUT and cnt.value == 0 and time.monotonic() - t0 >= 0.04
    # starting twice is refused; a stopped loop can be started again
    assert lib.hsma_server_start(srv.ptr) == -3
    srv.hsma_server_stop()
    srv.hsma_server_start()
    r = np.zeros(1, dtype=server.REQUEST)
    r["kind"] = server.REQ_ENERGY
    assert srv.hsma_server_submit(r[0]) == 0
    res = _poll_all(srv, 1)
    srv.hsma_server_stop()
    assert len(res) == 1 and res["status"][0] == 0 and res["ticket"][0] == 0
