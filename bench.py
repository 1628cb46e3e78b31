#!/usr/bin/env python
"""Benchmark of the GB300 HSMA hot path (arXiv:1907.01724, Algorithm 1 steps 4-5).

Headline workload: one cavity of N = 20000 unit charges uniform in a = 1, eps1 = eps2 = 78.5,
kappa a = 3, M = 2000 points per shell, p = 30 (the largest single-system workload).  One step =
the whole hot path (spatial order and Kelvin images, correction coefficients, surface images,
the tiled pair sum, the potential/energy reduction) as one CUDA-graph launch.  FP32 pair sums;
the moments, coefficients, surface synthesis and reductions in double-float arithmetic
(~2^-46 relative), the geometry of the records in FP64.

Metric: Coulomb pair-evaluations per second, counting per cavity N (2N - 1 + 3M) pairs (every
charge against the other real charges, the N Kelvin images and the 3M surface images of
eq. phicorrfinall).  Inputs are seeded synthetic data (random charges in the ball, the paper's
workload type).  L2 is flushed (256 MB write) before every timed step, outside the timed events.

Sections: the near-interface workload (two cavities of N = 2000, 25% within 0.05a of the
interface, M = 1000, p = 20), fields, the batched workload (512 cavities) and the serving loop.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own independent cavities (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1907_01724_gb300 import inputs  # noqa: E402

SM_MUFU_PER_CLK = 16  # rsqrt results per SM per clock (one pair evaluation each)
METRIC = "Coulomb pair-evals/s at rel err <=1e-6 vs FP64"
DTYPE = "f32 pair sums; double-float (~2^-46) moments, coefficients, surface and reductions; f64 geometry"


def workload(rank: int):
    """The headline workload: one cavity, N = 20000 uniform, eps1 = eps2 = 78.5, kappa a = 3,
    M = 2000, p = 30."""
    return [inputs.primitive_system(seed_offset=1000 * rank)]


def near_interface_workload(rank: int):
    off = 1000 * rank
    return [inputs.near_interface_system(kappa_a=0.5, seed_offset=off),
            inputs.near_interface_system(kappa_a=2.0, seed_offset=off)]


def pairs(s) -> int:
    return s.n * (2 * s.n - 1 + 3 * s.M)


def evals(s) -> int:
    """Kernel pair evaluations (one rsqrt each): a surface point carries monopole + dipole."""
    return s.n * (2 * s.n - 1 + s.M)


# the sources of the FP32 pair kernel, in the order its committed ncu summary hashes them
PAIR_KERNEL_SOURCES = ("k_pairs.cu", "k_pairs_f32.cuh", "pair_work.cuh", "fp32_pair.cuh", "df64.cuh",
                       "hsma_internal.cuh")


def kernel_source_sha(paths) -> str:
    """sha256 of the concatenated sources of a kernel (recorded with each committed ncu summary)."""
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        h.update(open(p, "rb").read())
    return h.hexdigest()


def profiled_traffic(kernel_srcs, profile_md: str):
    """DRAM bytes per launch from the committed ncu summary, or None if the kernel's source has
    changed since that capture (the summary records the source hash it was taken with)."""
    import re
    try:
        text = open(profile_md).read()
        sha = re.search(r"source_sha256 \([^)]*\): ([0-9a-f]+)", text).group(1)
        traffic = int(re.search(r"traffic_bytes_per_launch: (\d+)", text).group(1))
        cur = kernel_source_sha(kernel_srcs)[:len(sha)]
    except (OSError, AttributeError):
        return None
    return traffic if cur == sha else None


def config_dict(systems, n_gpus):
    s = systems[0]
    return {"workload": f"1 cavity N={s.n} uniform in a=1, eps1=eps2=78.5, kappa*a=3, M={s.M}, p={s.p}, "
                        f"tau=0.1, FP32 pair sums",
            "systems_per_gpu": len(systems), "N": s.n, "M": s.M, "p": s.p, "kappa_a": s.kappa * s.a,
            "eps1": s.eps1, "eps2": s.eps2,
            "pairs_per_step_per_gpu": int(sum(pairs(x) for x in systems)),
            "l2": "flushed before every timed step (256 MB write)", "parallelism": f"replicas x{n_gpus}"}


def affinity():
    """Host cores this process may run on: count and the mask as ranges."""
    try:
        cpus = sorted(os.sched_getaffinity(0))
    except AttributeError:
        cpus = list(range(os.cpu_count() or 1))
    rng, start, prev = [], None, None
    for c in cpus:
        if start is None:
            start = prev = c
        elif c == prev + 1:
            prev = c
        else:
            rng.append(f"{start}-{prev}" if prev > start else f"{start}")
            start = prev = c
    if start is not None:
        rng.append(f"{start}-{prev}" if prev > start else f"{start}")
    return len(cpus), ",".join(rng)


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce(world, x: float, op: str, device: str = "cuda") -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def aggregate(world: int, local_seconds: float, local_units: float, device: str = "cuda"):
    """Whole-job throughput over ranks: units of all ranks / the slowest rank's time."""
    t_max = allreduce(world, local_seconds, "max", device)
    units = allreduce(world, local_units, "sum", device)
    return units / t_max, t_max, units


def oracle_run(systems, budget_s: float = 10.0, max_rounds: int = 50, nthreads: int = 0):
    """FP64 oracle over the whole workload (build + potentials + energies of every system),
    repeated until about budget_s of CPU work; nthreads OpenMP threads (0 = one per core of the
    affinity mask).  Returns the results of the first round, pair-evals/s, seconds, rounds and
    the threads used."""
    import oracle
    th = nthreads if nthreads > 0 else affinity()[0]
    t0 = time.perf_counter()
    done = 0
    rounds = 0
    refs = None
    while True:
        out = []
        for s in systems:
            P = oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau,
                                   nthreads=th)
            out.append(oracle.hsma(P, s.xyz, s.q))
            done += pairs(s)
        refs = refs or out
        rounds += 1
        el = time.perf_counter() - t0
        if el >= budget_s or rounds >= max_rounds:
            break
    return refs, done / el, el, rounds, th


def cpu_baselines(systems, quick: bool):
    """The oracle timed on the host cores on the same workload: every core of the affinity mask
    (repeated to about 8 s), then one thread (one pass over the whole workload)."""
    ncores, mask = affinity()
    refs, rate, el, rounds, th = oracle_run(systems, budget_s=0.0 if quick else 8.0, max_rounds=1 if quick else 20)
    cpu = {"value": rate, "unit": "pair-evals/s", "cores": th, "kind": "oracle",
           "sample": f"whole workload (build + potentials + energies) x{rounds}, {el:.1f} s",
           "affinity": {"cores": ncores, "mask": mask}}
    if not quick:
        _, rate1, el1, rounds1, _ = oracle_run(systems, budget_s=0.0, max_rounds=1, nthreads=1)
        cpu["single_thread"] = {"value": rate1, "unit": "pair-evals/s", "cores": 1,
                                "sample": f"whole workload x{rounds1}, {el1:.1f} s"}
        cpu["batched_extrapolated"], cpu["serving_extrapolated"] = oracle_extrapolated(th)
        cpu["far_field_sampled"] = oracle_far_field_sample(th)
    return refs, cpu


_FAR_REF = {}  # sampled oracle potentials of the far-field workload (filled by the CPU leg)


def oracle_far_field_sample(th: int, n: int = 1_000_000, samples: int = 500):
    """The oracle on the far-field workload: its whole source build (Kelvin images, the
    correction series at the 3M surface points, O(N M p)) and the potentials at `samples` seeded
    charges (2N + 3M sources each); the far-field section compares the tree with them."""
    import oracle

    from paper_1907_01724_gb300 import inputs
    s = inputs.far_field_system(n)
    P = oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau, nthreads=th)
    t0 = time.perf_counter()
    src = oracle.build_sources(P, s.xyz, s.q)
    tb = time.perf_counter() - t0
    idx = np.sort(np.random.default_rng(13).choice(s.n, samples, replace=False))
    t0 = time.perf_counter()
    pc, pr = oracle.evaluate(P, s.xyz, s.q, src, s.xyz[idx], self_index=idx)
    te = time.perf_counter() - t0
    _FAR_REF[n] = (idx, pc + pr)
    return {"kind": "oracle", "cores": th,
            "sample": f"N={s.n}: whole source build {tb:.1f} s, then {samples} seeded charges' potentials "
                      f"against the {2 * s.n + 3 * s.M} sources {te:.2f} s",
            "value": samples * (2 * s.n - 1 + 3 * s.M) / te, "unit": "pair-evals/s (the sampled potentials)",
            "build_s": tb}


def oracle_extrapolated(th: int):
    """The oracle on seeded random subsets of the batched and serving workloads, scaled to the
    whole workload by pair count (labelled extrapolated): 8 of the 512 cavities; 4 of the 64
    chains with N <= 8000, with the request mix's mean pairs per request (a full energy is one
    whole-method evaluation; a move's energy change is two, as the oracle defines it)."""
    import oracle

    from paper_1907_01724_gb300 import inputs
    rng = np.random.default_rng(11)
    bs = inputs.batched_systems()
    idx = sorted(rng.choice(len(bs), 8, replace=False).tolist())
    t0 = time.perf_counter()
    for i in idx:
        s = bs[i]
        oracle.hsma(oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau,
                                       nthreads=th), s.xyz, s.q)
    tb = time.perf_counter() - t0
    ps, pa = sum(pairs(bs[i]) for i in idx), sum(pairs(s) for s in bs)
    batched = {"kind": "oracle, extrapolated by pair count", "cores": th,
               "sample": f"cavities {idx} of {len(bs)} ({ps:.3g} of {pa:.3g} pairs), {tb:.2f} s",
               "pair_evals_per_s": ps / tb, "systems_per_s": len(bs) / (tb * pa / ps)}
    wl = inputs.serving_workload()
    small = [c for c in range(len(wl.chains)) if wl.chains[c].n <= 8000]
    cs = sorted(rng.choice(small, 4, replace=False).tolist())
    t0 = time.perf_counter()
    for c in cs:
        s = wl.chains[c]
        oracle.hsma(oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau,
                                       nthreads=th), s.xyz, s.q)
    tsv = time.perf_counter() - t0
    rate = sum(pairs(wl.chains[c]) for c in cs) / tsv
    per_req = sum(pairs(s) for s in wl.chains) / len(wl.chains) * (wl.frac_delta * 2 + (1 - wl.frac_delta))
    serving = {"kind": "oracle, extrapolated by pair count", "cores": th,
               "sample": f"chains {cs} (N <= 8000) of {len(wl.chains)}, one evaluation each, {tsv:.2f} s",
               "pair_evals_per_s": rate, "mean_pairs_per_request": per_req, "req_per_s": rate / per_req}
    return batched, serving


def accuracy(systems, refs, phi, et):
    """Norm-wise potential errors, pointwise maxima and energy errors against the oracle."""
    out = {"phi_rel_l2_max": 0.0, "phi_pointwise_abs_over_max": 0.0, "energy_rel_max": 0.0,
           "reference": "FP64 oracle"}
    off = 0
    for s, r, e in zip(systems, refs, et):
        p = phi[off:off + s.n]
        off += s.n
        d = np.abs(p - r["phi"])
        scale = max(abs(r["E_total"]), 0.5 * float(np.sum(np.abs(s.q * r["phi"]))))
        out["phi_rel_l2_max"] = max(out["phi_rel_l2_max"], float(np.linalg.norm(d) / np.linalg.norm(r["phi"])))
        out["phi_pointwise_abs_over_max"] = max(out["phi_pointwise_abs_over_max"],
                                                float(d.max() / np.abs(r["phi"]).max()))
        out["energy_rel_max"] = max(out["energy_rel_max"], abs(e - r["E_total"]) / scale)
    return out


def timed_steps(step, stream, flush, k):
    """k steps, L2 flushed before each (outside the events), CUDA events on the work stream;
    returns the total seconds."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    for i in range(k):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(c) for a, c in ev) / 1e3


def pair_kernel_alone(b, step, flush, reps):
    """The pair kernel timed alone: in the timed steps it runs in one graph with the build, so it
    is timed in separate passes (same items, bitwise the same results), CUDA events around each
    launch on its stream; mean seconds per launch."""
    b.hsma_batch_set_overlap(False)
    ms = []
    for _ in range(reps):
        flush.zero_()
        step()
        ms.append(b.hsma_batch_last_pair_time())
    b.hsma_batch_set_overlap(True)
    return statistics.mean(ms) / 1e3, len(ms)


def e2e_run(b, n, xyz, q, units_per_step, world, k):
    """End to end through the C ABI with pinned host buffers: the host-to-device transfer of the
    inputs (read in place from the page-locked arrays by the pass's first kernels), the step, and
    the device-to-host transfer of the potentials (written into a page-locked array by the
    reduction) and of the energies, all inside the timed region."""
    import torch

    from paper_1907_01724_gb300 import api
    xyz_h = torch.tensor(xyz).pin_memory().numpy()
    q_h = torch.tensor(q).pin_memory().numpy()
    phi_h = torch.empty(int(n.sum()), dtype=torch.float64).pin_memory().numpy()

    def e2e_step():
        b.hsma_batch_build_sources(n, xyz_h, q_h)
        b.hsma_batch_potential(api.HSMA_TOTAL, out=phi_h)
        b.hsma_batch_energy()

    for _ in range(3):
        e2e_step()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k):
        e2e_step()
    torch.cuda.synchronize()
    te = allreduce(world, time.perf_counter() - t0, "max")
    return {"value": allreduce(world, float(units_per_step * k), "sum") / te,
            "unit": "pair-evals/s", "h2d_bytes_per_step": int(32 * n.sum()),
            "d2h_bytes_per_step": int(8 * n.sum() + 16 * len(n)), "steps": k,
            "ms_per_step": te / k * 1e3}


def run_near_interface(local, stream, gpu_name, steps):
    """The near-interface workload (two cavities of N = 2000, 25% within 0.05a of the interface,
    M = 1000, p = 20): whole-path steps, the pair kernel alone, end to end, accuracy."""
    import torch

    from paper_1907_01724_gb300 import api, batch
    systems = near_interface_workload(0)
    refs, _, _, _, _ = oracle_run(systems, budget_s=0.0, max_rounds=1)
    n, xyz, q = batch.concat(systems)
    b = batch.from_systems(systems, precision=api.HSMA_FP32, device=local, stream=stream)
    cfg = batch.autotuned(b, n, xyz, q, gpu=gpu_name, reps=5)
    dev = torch.device(f"cuda:{local}")
    xyz_d = torch.tensor(xyz, device=dev)
    q_d = torch.tensor(q, device=dev)
    phi_d = torch.empty(int(n.sum()), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        b.hsma_batch_build_sources(n, xyz_d, q_d)
        b.hsma_batch_potential(api.HSMA_TOTAL, out=phi_d)

    for _ in range(20):
        step()
    torch.cuda.synchronize()
    acc = accuracy(systems, refs, b.hsma_batch_potential(api.HSMA_TOTAL), b.hsma_batch_energy()[0])
    k = max(200, steps)
    t = timed_steps(step, stream, flush, k)
    units = sum(pairs(s) for s in systems)
    t_pair, nrep = pair_kernel_alone(b, step, flush, 100)
    props = torch.cuda.get_device_properties(local)
    peak = props.multi_processor_count * SM_MUFU_PER_CLK * 2070.0e6
    e2e = e2e_run(b, n, xyz, q, units, 1, max(50, steps // 4))
    return {"workload": "2 cavities N=2000 (25% within 0.05a of the interface), eps1=1, eps2=80, "
                        "kappa*a in {0.5,2}, M=1000, p=20, tau=0.1, FP32 pair sums",
            "value": units * k / t, "unit": "pair-evals/s", "ms_per_step": t / k * 1e3, "steps": k,
            "pair_kernel_alone": {"ms": t_pair * 1e3, "launches": nrep,
                                  "frac_of_mufu_peak_at_2070MHz": units / t_pair / peak,
                                  "frac_kernel_evals": sum(evals(s) for s in systems) / t_pair / peak},
            "e2e": e2e, "pair_config": batch.pair_configs()[cfg], "pair_schedule": b.hsma_batch_pair_schedule(),
            "accuracy_vs_oracle": acc,
            "l2": "flushed before every timed step (256 MB write)"}


def run_far_field(local, stream, steps: int = 5, theta: float = 0.5, order: int = 12, n: int = 1_000_000,
                  smaller: int | None = 200_000):
    """The paper's N = 1e6 timing workload (Sec. 4.2: p = 20, F1/F2 = 987/1597) with the
    treecode far field (hsma_set_far_field) against the direct pair sum on the same GPU: whole
    build + potential steps from device inputs (L2 flushed before each, CUDA events), the tree's
    evaluation kernel alone, and the norm-wise difference of the two FP32 results; the same at
    N = `smaller` (its `smaller` entry) for the trend with N."""
    import torch

    from paper_1907_01724_gb300 import api, inputs
    s = inputs.far_field_system(n)
    dev = torch.device(f"cuda:{local}")
    xyz_d = torch.tensor(s.xyz, device=dev)
    q_d = torch.tensor(s.q, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    units = pairs(s)
    res = {"workload": f"1 cavity N={s.n} uniform in a=1, eps1=2, eps2=80, kappa*a=5, p=20, F1/F2=987/1597 "
                       f"(M={s.M}), tau=0.1 (the paper's timing workload, Sec. 4.2)",
           "pairs_per_step": units}
    phis = {}
    for label, th in (("tree", theta), ("direct", 0.0)):
        prm = api.hsma_default_params(p=s.p, M=s.M, tau=s.tau, precision=api.HSMA_FP32, device=local,
                                      stream=stream.cuda_stream)
        h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
        if th > 0:
            api.hsma_set_far_field(h, th, order)
        phi_d = torch.empty(s.n, dtype=torch.float64, device=dev)

        def step():
            api.hsma_build_sources(h, xyz_d, q_d)
            api.hsma_potential(h, api.HSMA_TOTAL, out=phi_d)

        k = steps if th > 0 else max(2, steps // 2)
        for _ in range(2):
            step()
        torch.cuda.synchronize()
        t = timed_steps(step, stream, flush, k)
        entry = {"ms_per_step": t / k * 1e3, "steps": k, "pair_evals_per_s": units * k / t}
        if th > 0:
            entry.update({"theta": th, "order": order, "eval_kernel_ms": api.hsma_last_far_time(h),
                          "kernel": "k_tree_eval"})
        phis[label] = phi_d.cpu().numpy()
        res[label] = entry
        api.hsma_destroy(h)
        del phi_d
        torch.cuda.empty_cache()
    d = phis["tree"] - phis["direct"]
    res["speedup_vs_direct"] = res["direct"]["ms_per_step"] / res["tree"]["ms_per_step"]
    res["tree_vs_direct_rel_l2"] = float((d @ d) ** 0.5 / (phis["direct"] @ phis["direct"]) ** 0.5)
    if n in _FAR_REF:
        idx, ref = _FAR_REF[n]
        for label in ("tree", "direct"):
            e = phis[label][idx] - ref
            res[label]["rel_l2_vs_oracle_sampled"] = float((e @ e) ** 0.5 / (ref @ ref) ** 0.5)
        res["oracle_sample"] = f"{len(idx)} seeded charges (the CPU leg's far_field_sampled)"
    res["paper_context"] = "HSMA + FMM, N = 1e6: 24 s on 32 cores of 4x Opteron 6272 (Sec. 4.2); not the target"
    if smaller:
        sm = run_far_field(local, stream, steps, theta, order, n=smaller, smaller=None)
        res["smaller"] = {k: sm[k] for k in ("workload", "tree", "direct", "speedup_vs_direct",
                                             "tree_vs_direct_rel_l2")}
    return res


def run_tree_only(local, stream, n: int, steps: int, theta: float = 0.5, order: int = 12):
    """The far-field workload's charges at N = n with the treecode, the build and the potential
    pass in separate graphs, `steps` passes (for profiling the tree's kernels)."""
    import torch

    from paper_1907_01724_gb300 import api, inputs
    s = inputs.far_field_system(n)
    prm = api.hsma_default_params(p=s.p, M=s.M, tau=s.tau, precision=api.HSMA_FP32, device=local,
                                  stream=stream.cuda_stream)
    h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
    api.hsma_set_far_field(h, theta, order)
    api.hsma_set_overlap(h, False)
    ms = []
    for _ in range(steps):
        api.hsma_build_sources(h, s.xyz, s.q)
        api.hsma_potential(h, api.HSMA_TOTAL)
        ms.append(api.hsma_last_far_time(h))
    api.hsma_destroy(h)
    torch.cuda.synchronize()
    return {"workload": s.name, "theta": theta, "order": order, "passes": steps, "eval_kernel_ms": ms}


def run_batched(local, stream, gpu_name):
    """512 independent cavities (N log-uniform in [100, 1e4]) in one batch: build + potentials +
    energies per launch pair; requests = systems evaluated.  Compared with the plain FP64
    single-system path (one handle per system, sequential) on a seeded subset, scaled by pairs."""
    import torch

    from paper_1907_01724_gb300 import api, batch
    systems = inputs.batched_systems()
    n, xyz, q = batch.concat(systems)
    b = batch.from_systems(systems, device=local, stream=stream)
    cfg = batch.autotuned(b, n, xyz, q, gpu=gpu_name, reps=3)
    xyz_d = torch.tensor(xyz, device=f"cuda:{local}")
    q_d = torch.tensor(q, device=f"cuda:{local}")
    phi_d = torch.empty(int(n.sum()), dtype=torch.float64, device=f"cuda:{local}")
    for _ in range(2):
        b.hsma_batch_build_sources(n, xyz_d, q_d)
        b.hsma_batch_potential(api.HSMA_TOTAL, out=phi_d)
    torch.cuda.synchronize()
    k = 5
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k):
        b.hsma_batch_build_sources(n, xyz_d, q_d)
        b.hsma_batch_potential(api.HSMA_TOTAL, out=phi_d)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    tot_pairs = sum(pairs(s) for s in systems)
    # the pair kernel alone (separate passes), for its roofline at this size
    b.hsma_batch_set_overlap(False)
    kern = []
    for _ in range(3):
        b.hsma_batch_build_sources(n, xyz_d, q_d)
        b.hsma_batch_potential(api.HSMA_TOTAL, out=phi_d)
        kern.append(b.hsma_batch_last_pair_time())
    b.hsma_batch_set_overlap(True)
    t_kern = statistics.median(kern) / 1e3
    props = torch.cuda.get_device_properties(local)
    peak = props.multi_processor_count * SM_MUFU_PER_CLK * 2070.0e6
    kern_evals = sum(evals(s) for s in systems) / t_kern
    et, _ = b.hsma_batch_energy()
    # accuracy on a seeded sample against the oracle
    import oracle
    rng = np.random.default_rng(7)
    sample = sorted(rng.choice(len(systems), 4, replace=False).tolist())
    worst = 0.0
    for i in sample:
        s = systems[i]
        P = oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M)
        r = oracle.hsma(P, s.xyz, s.q)
        scale = max(abs(r["E_total"]), 0.5 * float(np.sum(np.abs(s.q * r["phi"]))))
        worst = max(worst, abs(et[i] - r["E_total"]) / scale)
    # plain FP64 single-system path on a seeded subset of 16 systems
    sub = sorted(rng.choice(len(systems), 16, replace=False).tolist())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in sub:
        s = systems[i]
        prm = api.hsma_default_params(p=s.p, M=s.M, tau=s.tau, precision=api.HSMA_FP64, device=local)
        h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
        api.hsma_build_sources(h, s.xyz, s.q)
        api.hsma_energy(h)
    t64 = time.perf_counter() - t0
    sub_pairs = sum(pairs(systems[i]) for i in sub)
    fp64_req_s = len(sub) / t64
    fp64_pairs_s = sub_pairs / t64
    return {"workload": f"{len(systems)} cavities, N log-uniform [100, 1e4] (sum {int(n.sum())}), a~U[0.8,1.5], "
                        "kappa*a~U[0.5,3], eps1 in {1, 78.5}, eps2=78.5, M=1000, p=20",
            "req_per_s": len(systems) * k / t, "pair_evals_per_s": tot_pairs * k / t, "ms_per_batch": t / k * 1e3,
            "pair_config": batch.pair_configs()[cfg], "pair_schedule": b.hsma_batch_pair_schedule(),
            "energy_rel_err_max_vs_oracle_sample": worst,
            "pair_kernel_alone": {"ms": t_kern * 1e3, "evals_per_s": kern_evals,
                                  "frac_of_mufu_peak_at_2070MHz": kern_evals / peak},
            "fp64_single_system": {"req_per_s": fp64_req_s, "pair_evals_per_s": fp64_pairs_s,
                                   "sample": "16 seeded systems, one FP64 handle each, host inputs"}}


def run_field(local, stream, systems, gpu_name):
    """Fields and potentials in one pass (hsma_batch_field) on the near-interface workload: build +
    field per step, the field pass's pair-evals/s, its kernel alone, and E against the oracle."""
    import torch

    from paper_1907_01724_gb300 import api, batch
    n, xyz, q = batch.concat(systems)
    b = batch.from_systems(systems, precision=api.HSMA_FP32, device=local, stream=stream)
    cfg = batch.autotuned(b, n, xyz, q, gpu=gpu_name, reps=3)
    xyz_d = torch.tensor(xyz, device=f"cuda:{local}")
    q_d = torch.tensor(q, device=f"cuda:{local}")
    E_d = torch.empty((int(n.sum()), 3), dtype=torch.float64, device=f"cuda:{local}")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    for _ in range(5):
        b.hsma_batch_build_sources(n, xyz_d, q_d)
        b.hsma_batch_field(api.HSMA_TOTAL, out=E_d)
    torch.cuda.synchronize()
    k = 500
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    for i in range(k):
        flush.zero_()
        ev[i][0].record(stream)
        b.hsma_batch_build_sources(n, xyz_d, q_d)
        b.hsma_batch_field(api.HSMA_TOTAL, out=E_d)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    t = sum(a.elapsed_time(c) for a, c in ev) / 1e3
    # the field kernel alone: in the timed steps it runs in one graph with the build, so it is
    # timed in separate passes (same items), events around each launch
    b.hsma_batch_set_overlap(False)
    kern = []
    for _ in range(50):
        flush.zero_()
        b.hsma_batch_build_sources(n, xyz_d, q_d)
        b.hsma_batch_field(api.HSMA_TOTAL, out=E_d)
        kern.append(b.hsma_batch_last_pair_time())
    b.hsma_batch_set_overlap(True)
    E = E_d.cpu().numpy()
    import oracle
    worst, off = 0.0, 0
    for s in systems:
        P = oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau)
        ref = oracle.field(P, s.xyz, s.q)["E"]
        worst = max(worst, float(np.linalg.norm(E[off:off + s.n] - ref) / np.linalg.norm(ref)))
        off += s.n
    tk = statistics.mean(kern) / 1e3
    ev_per_launch = sum(evals(s) for s in systems)
    return {"workload": "the near-interface workload, fields and potentials in one pass (build + field per step)",
            "pair_evals_per_s": sum(pairs(s) for s in systems) * k / t, "ms_per_step": t / k * 1e3, "steps": k,
            "field_kernel_ms": tk * 1e3, "field_kernel_evals_per_s": ev_per_launch / tk,
            "pair_config": batch.pair_configs()[cfg], "E_rel_l2_max_vs_oracle": worst,
            "l2": "flushed before every timed step (256 MB write)"}


def run_serving(local):
    """64 Monte Carlo chains (N log-uniform in [500, 5e4]), 90% move / 10% full-energy requests.
    Saturation = all requests released at once; then Poisson arrivals at 0.25/0.5/0.8/0.95 of it."""
    from paper_1907_01724_gb300 import api, server
    wl = inputs.serving_workload()
    srv = server.Server(wl.chains, max_batch=64, energy_slots=4, energy_sm_frac=0.75, device=local)
    srv.hsma_server_load()
    pos = [c.xyz.copy() for c in wl.chains]
    # warm-up and saturation
    reqs, pos = server.make_trace(wl, 500, None, pos)
    srv.hsma_server_run(reqs)
    reqs, pos = server.make_trace(wl, 3000, None, pos)
    res = srv.hsma_server_run(reqs)
    sat = server.latency_stats(res, reqs)
    out = {"workload": "64 chains, N log-uniform [500, 5e4] (sum %d), M=1000, p=20; 90%% single-move dE "
                       "(commit with p=0.5), 10%% full energies" % sum(c.n for c in wl.chains),
           "driver": "hsma_server_run: the calling thread submits each request at its release time through "
                     "hsma_server_submit and takes the answers through hsma_server_poll; the request loop "
                     "runs on its own native thread",
           "saturation": sat, "loads": {}}
    for f in (0.25, 0.5, 0.8, 0.95):
        rate = f * sat["req_per_s"]
        nreq = int(min(20000, max(300, rate * 1.0)))
        reqs, pos = server.make_trace(wl, nreq, rate, pos)
        res = srv.hsma_server_run(reqs)
        st = server.latency_stats(res, reqs)
        st["offered_req_per_s"] = rate
        out["loads"][str(f)] = st
    # plain FP64 single-system path: the same kind of requests, one handle per chain, sequential
    rng = np.random.default_rng(11)
    lat = []
    for c in sorted(rng.choice(len(wl.chains), 4, replace=False).tolist()):
        ch = wl.chains[c]
        prm = api.hsma_default_params(p=ch.p, M=ch.M, tau=ch.tau, precision=api.HSMA_FP64, device=local)
        h = api.hsma_create(ch.a, ch.eps1, ch.eps2, ch.kappa, prm)
        api.hsma_build_sources(h, ch.xyz, ch.q)
        api.hsma_energy(h)
        for j in range(10):
            k = int(rng.integers(ch.n))
            x = ch.xyz[k] * 0.98
            t0 = time.perf_counter()
            if j % 10 == 9:
                api.hsma_build_sources(h, ch.xyz, ch.q)
                api.hsma_energy(h)
            else:
                api.hsma_delta_energy(h, k, x)
            lat.append(time.perf_counter() - t0)
    lat = np.array(lat)
    out["fp64_single_system"] = {"p50_ms": float(np.percentile(lat, 50) * 1e3),
                                 "p99_ms": float(np.percentile(lat, 99) * 1e3),
                                 "req_per_s": float(len(lat) / lat.sum()),
                                 "sample": "40 requests (9 moves : 1 full energy) on 4 seeded chains, sequential"}
    return out


def run_ours(args):
    import torch

    from paper_1907_01724_gb300 import api, batch

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    systems = workload(rank)

    # oracle baseline first (rank 0), before any GPU timing; its results also check accuracy
    cpu = None
    refs = None
    if rank == 0:
        refs, cpu = cpu_baselines(systems, quick=args.no_cpu_baseline or world > 1)
        if world > 1:
            cpu = None

    n, xyz, q = batch.concat(systems)
    b = batch.from_systems(systems, precision=api.HSMA_FP32, device=local, stream=stream)
    gpu_name = torch.cuda.get_device_name(local)
    cfg = batch.autotuned(b, n, xyz, q, gpu=gpu_name, reps=5)
    xyz_d = torch.tensor(xyz, device=dev)
    q_d = torch.tensor(q, device=dev)
    phi_d = torch.empty(int(n.sum()), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        b.hsma_batch_build_sources(n, xyz_d, q_d)
        b.hsma_batch_potential(api.HSMA_TOTAL, out=phi_d)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    acc = None
    if refs is not None:
        acc = accuracy(systems, refs, b.hsma_batch_potential(api.HSMA_TOTAL), b.hsma_batch_energy()[0])

    units = sum(pairs(s) for s in systems)
    launches0 = b.hsma_batch_kernel_launches()
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    t_local = timed_steps(step, stream, flush, args.steps)
    clk = clocks.stop()
    barrier(world)
    launches = b.hsma_batch_kernel_launches() - launches0
    value, t_max, total_pairs = aggregate(world, t_local, float(units * args.steps))

    # dominant kernel alone: algorithmic pairs per launch (N (2N - 1 + 3M) per cavity) / the
    # event-timed launch duration
    t_pair, nrep = pair_kernel_alone(b, step, flush, max(20, min(200, args.steps)))
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak = sms * SM_MUFU_PER_CLK * sm_max * 1e6
    achieved = units / t_pair
    ev_per_launch = sum(evals(s) for s in systems)
    csrc = os.path.join(ROOT, "paper_1907_01724_gb300", "csrc")
    traffic = profiled_traffic([os.path.join(csrc, f) for f in PAIR_KERNEL_SOURCES],
                               os.path.join(ROOT, "profiles", "k_pairs_f32_N20000_M2000_p30.md"))
    roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair-eval/s",
            "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch (ncu dram read+write)",
            "kernel": "k_pairs_f32",
            "work_unit": "pairs N(2N-1+3M) per cavity per launch (a surface point's monopole and two dipole "
                         "charges count 3)",
            "peak_basis": f"{sms} SMs x {SM_MUFU_PER_CLK} MUFU rsqrt/clk x {sm_max:.0f} MHz (max SM clock)",
            "frac_kernel_evals": ev_per_launch / t_pair / peak,
            "kernel_evals_note": "N(2N-1+M) evaluations per cavity: one rsqrt per pair, a surface point's "
                                 "monopole and dipole share one",
            "unique_rsqrt_per_launch": sum(s.n * s.n + s.n * s.M for s in systems),
            "frac_unique_rsqrt": sum(s.n * s.n + s.n * s.M for s in systems) / t_pair / peak,
            "unique_rsqrt_note": "the rsqrt evaluations the kernel needs: real and Kelvin pairs once per unordered "
                                 "pair (Newton's third law; Kelvin inversion), N(N-1)/2 + N(N+1)/2 + NM per cavity "
                                 "(+ ~1% for the one-way diagonal blocks): the MUFU's own utilisation",
            "pair_kernel_ms": t_pair * 1e3, "pair_config": batch.pair_configs()[cfg], "pair_config_index": cfg,
            "pair_schedule": b.hsma_batch_pair_schedule(),
            "pairs_per_launch": units,
            "timing": f"{nrep} launches in separate passes (L2 flushed before each step), CUDA events "
                      "on the launch stream; in the timed steps the kernel runs in one graph with the "
                      "build (order and records beside the coefficient chain, then the pair sum)"}
    if clk.get("sm_mhz"):
        roof["frac_at_median_clock"] = achieved / (sms * SM_MUFU_PER_CLK * clk["sm_mhz"] * 1e6)

    # plain FP64 path on the same GPU (comparator)
    b64 = batch.from_systems(systems, precision=api.HSMA_FP64, device=local, stream=stream)
    b64.hsma_batch_build_sources(n, xyz, q)

    def step64():
        b64.hsma_batch_build_sources(n, xyz_d, q_d)
        b64.hsma_batch_potential(api.HSMA_TOTAL, out=phi_d)

    step64()
    torch.cuda.synchronize()
    k64 = 3
    t64 = timed_steps(step64, stream, flush, k64)
    fp64 = {"value": units * k64 / t64, "unit": "pair-evals/s", "ms_per_step": t64 / k64 * 1e3, "steps": k64}
    del b64

    e2e = e2e_run(b, n, xyz, q, units, world, max(10, args.steps))

    near = batched = serving = fieldres = far = None
    if rank == 0 and world == 1 and not args.no_extras:
        near = run_near_interface(local, stream, gpu_name, args.steps)
        fieldres = run_field(local, stream, near_interface_workload(0), gpu_name)
        batched = run_batched(local, stream, gpu_name)
        serving = run_serving(local)
        far = run_far_field(local, stream)
        if cpu is not None:
            batched["oracle_extrapolated"] = cpu.get("batched_extrapolated")
            serving["oracle_extrapolated"] = cpu.get("serving_extrapolated")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "pair-evals/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE,
                "data": "synthetic (seeded random charges uniform in the ball)",
                "config": config_dict(systems, world), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk, "gpu_launches": int(launches), "accuracy_vs_oracle": acc, "fp64_path": fp64,
                "near_interface": near, "field": fieldres, "batched": batched, "serving": serving,
                "far_field": far,
                "impl": "ours"}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    systems = workload(0)
    th, mask = affinity()

    def one_step():
        for s in systems:
            P = oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau,
                                   nthreads=th)
            oracle.hsma(P, s.xyz, s.q)

    # warm-up: one full pass (also measures the cost of a step)
    t0 = time.perf_counter()
    one_step()
    t_step = time.perf_counter() - t0
    k = int(max(1, min(args.steps, math.ceil(60.0 / max(t_step, 1e-3)))))
    t0 = time.perf_counter()
    for _ in range(k):
        one_step()
    el = time.perf_counter() - t0
    value = sum(pairs(s) for s in systems) * k / el
    line = {"metric": METRIC, "value": value, "unit": "pair-evals/s", "n_gpus": world, "steps": k,
            "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": el / k * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded random charges uniform in the ball)",
            "config": config_dict(systems, 1), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "pair-evals/s", "kind": "oracle", "cores": th,
                             "affinity": {"cores": th, "mask": mask},
                             "sample": f"whole workload (build + potentials + energies) x{k} steps, "
                                       "bounded to about 60 s"},
            "e2e": {"value": value, "unit": "pair-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the near-interface, field, batched and "
                                                             "serving sections")
    ap.add_argument("--pair-config", type=int, default=-1,
                    help="with --only pairs / steps / near_steps: this tile configuration (index of "
                         "batch.pair_configs()) instead of the autotuned one")
    ap.add_argument("--pair-schedule", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="with --only steps / near_steps and --pair-config: the real/Kelvin pair schedule "
                         "(1 beside the coefficient chain, 2 the same leaving room for a coefficient or "
                         "surface CTA per SM, 0 after it; -1 the library's default)")
    ap.add_argument("--only", choices=["batched", "serving", "field", "near", "pairs", "steps", "near_steps",
                                       "far", "tree"],
                    help="run one section alone (profiling); 'pairs': the headline workload's pair kernel "
                         "in separate passes (--steps launches); 'steps' / 'near_steps': --warmup + --steps "
                         "whole-path steps of the headline / near-interface workload and nothing else")
    ap.add_argument("--far-n", type=int, default=1_000_000,
                    help="with --only tree: charges of the far-field workload")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.only:
        import torch
        torch.cuda.set_device(0)
        st = torch.cuda.Stream()
        torch.cuda.set_stream(st)
        name = torch.cuda.get_device_name(0)
        if args.only == "batched":
            out = run_batched(0, st, name)
        elif args.only == "field":
            out = run_field(0, st, near_interface_workload(0), name)
        elif args.only == "near":
            out = run_near_interface(0, st, name, args.steps)
        elif args.only == "far":
            out = run_far_field(0, st, steps=args.steps)
        elif args.only == "tree":
            out = run_tree_only(0, st, args.far_n, args.steps)
        elif args.only == "pairs":
            out = run_pairs_only(0, st, name, args.steps, args.warmup, args.pair_config)
        elif args.only in ("steps", "near_steps"):
            wl = workload(0) if args.only == "steps" else near_interface_workload(0)
            out = run_steps_only(0, st, name, wl, args.steps, args.warmup, args.pair_config, args.pair_schedule)
        else:
            out = run_serving(0)
        print(json.dumps(out), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


def run_pairs_only(local, stream, gpu_name, steps, warmup, pair_config=-1):
    """The headline workload with the build and the pair sum in separate passes: warmup + steps
    potential passes (for profiling the pair kernel; the launch list shows one k_pairs_f32 per
    pass)."""
    import torch

    from paper_1907_01724_gb300 import api, batch
    systems = workload(0)
    n, xyz, q = batch.concat(systems)
    b = batch.from_systems(systems, precision=api.HSMA_FP32, device=local, stream=stream)
    if pair_config >= 0:
        cfg = pair_config
        b.hsma_batch_set_pair_config(cfg)
    else:
        cfg = batch.autotuned(b, n, xyz, q, gpu=gpu_name, reps=5)
    b.hsma_batch_set_overlap(False)
    xyz_d = torch.tensor(xyz, device=f"cuda:{local}")
    q_d = torch.tensor(q, device=f"cuda:{local}")
    phi_d = torch.empty(int(n.sum()), dtype=torch.float64, device=f"cuda:{local}")
    ms = []
    for i in range(warmup + steps):
        b.hsma_batch_build_sources(n, xyz_d, q_d)
        b.hsma_batch_potential(api.HSMA_TOTAL, out=phi_d)
        if i >= warmup:
            ms.append(b.hsma_batch_last_pair_time())
    torch.cuda.synchronize()
    return {"workload": config_dict(systems, 1)["workload"], "pair_config": batch.pair_configs()[cfg],
            "pair_config_index": cfg,
            "pair_kernel_ms_mean": statistics.mean(ms) if ms else None, "launches": len(ms)}


def run_steps_only(local, stream, gpu_name, systems, steps, warmup, pair_config=-1, pair_schedule=-1):
    """warmup + steps whole-path steps (build + potentials in one graph) of a workload,
    device inputs, nothing else (for launch lists); the tile configuration and pair schedule
    given or autotuned."""
    import torch

    from paper_1907_01724_gb300 import api, batch
    n, xyz, q = batch.concat(systems)
    b = batch.from_systems(systems, precision=api.HSMA_FP32, device=local, stream=stream)
    if pair_config >= 0:
        cfg = pair_config
        b.hsma_batch_set_pair_config(cfg)
        b.hsma_batch_set_pair_schedule(pair_schedule)
    else:
        cfg = batch.autotuned(b, n, xyz, q, gpu=gpu_name, reps=5)
    xyz_d = torch.tensor(xyz, device=f"cuda:{local}")
    q_d = torch.tensor(q, device=f"cuda:{local}")
    phi_d = torch.empty(int(n.sum()), dtype=torch.float64, device=f"cuda:{local}")
    for _ in range(warmup + steps):
        b.hsma_batch_build_sources(n, xyz_d, q_d)
        b.hsma_batch_potential(api.HSMA_TOTAL, out=phi_d)
    torch.cuda.synchronize()
    return {"systems": len(systems), "N": [s.n for s in systems], "pair_config": batch.pair_configs()[cfg],
            "pair_config_index": cfg, "pair_schedule": b.hsma_batch_pair_schedule(), "steps": steps,
            "warmup": warmup}


if __name__ == "__main__":
    main()
