"""Benchmark: swap attempts per second of the checkerboard Metropolis sweep.

Workload (N=1): BCC 800^3 cubic cells = 1,024,000,000 sites, 4 species at
equiatomic composition, packed 4-bit storage, 4-shell EPI drawn from
N(0, 20 meV), 1200 K.  A step is one sweep (one swap trial per site) with
shared-direction proposals (one shell-1 direction per sweep, tile and phase;
acceptance uniforms per trial); `per_trial_direction` times the same sweep
with a direction drawn per trial.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  `value` is device-timed throughput with the lattice
resident in HBM; `e2e` repeats the measurement through the C ABI with the
configuration uploaded from pinned host memory every step and the energy read
back; `roofline` covers the sweep kernel; `cpu_baseline` times the serial CPU
oracle on a bounded sample of the same workload.  Under torchrun each rank
sweeps its own independent replica (weak scaling, no collective on the data
path).  `--impl reference` times the oracle alone (the reference arm).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2503_12591_gb300.inputs import (SCALE_BCC800, batched_edges, epi_gaussian, equiatomic,  # noqa: E402
                                           log_temperatures)

METRIC = "swap attempts/s at 1.02B-site BCC (HBM roofline %); batched & gradient vs plain"
UNIT = "attempts/s"
WORK = SCALE_BCC800
T_KELVIN = WORK.temperatures[0]
SEED = 1
# Proposal mode of the headline sweep: one shell-1 direction per (sweep, tile,
# intra colour), smcx PROPOSAL_TILE / oracle proposal 1.
PROPOSAL = 1
# Bytes of the lattice store a sweep must read and write per site (packed
# 4-bit: half a byte in, half a byte out).
ALG_BYTES_PER_ATTEMPT = 1.0
# Shared-memory lane loads per trial the method cannot avoid: the species of
# s and s' plus the 68 distinct sites of their 4-shell BCC environments.
ALG_GATHERS_PER_ATTEMPT = 70
SM_COUNT_NOMINAL = 152
SM_MAX_MHZ_NOMINAL = 2070.0
# CPU sample: same lattice kind, species, shells, temperature and schedule
# shape on a smaller box.
CPU_SAMPLE_DIMS = (64, 64, 64)
CPU_SAMPLE_SCHED = (3, (4, 4, 4))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="smcx", choices=["smcx", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-site", action="store_true", help="skip the per-trial-direction measurement")
    ap.add_argument("--no-clusters", action="store_true")
    ap.add_argument("--no-qsro", action="store_true")
    ap.add_argument("--no-throughput", action="store_true")
    ap.add_argument("--no-anneal", action="store_true")
    ap.add_argument("--no-fcc", action="store_true")
    ap.add_argument("--no-paper", action="store_true")
    ap.add_argument("--only", default="", choices=["", "batched", "exchange", "gradient", "clusters", "qsro",
                                                    "throughput", "anneal", "fcc", "paper", "baselines",
                                                    "batch_launch", "qsro_launch"],
                    help="profiling only: run one secondary measurement and print its JSON")
    ap.add_argument("--edge", type=int, default=0,
                    help="profiling only: lattice edge of the fcc / qsro / clusters measurement")
    ap.add_argument("--dims", type=int, default=0,
                    help="profiling only: cubic BCC edge other than the 800 of the workload")
    ap.add_argument("--proposal", type=int, default=1, choices=[0, 1, 2],
                    help="profiling only: proposal mode of the batch_launch measurement")
    ap.add_argument("--batch-sched", default="3,17,256",
                    help="profiling only: link cell, tile target and CTA threads of batch_launch")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(n_sweeps=24, n_serial=4):
    """The oracle as it stands on a BCC 64^3 sample: its OpenMP mode (each
    phase's sites split across all host cores, identical result) and, for
    reference, its serial mode."""
    import oracle as O

    V = epi_gaussian(WORK.K, WORK.M, WORK.sigma_mev, WORK.epi_seed)
    sig = O.init_config(O.BCC, CPU_SAMPLE_DIMS, WORK.M, equiatomic(WORK.M), WORK.init_seed)
    t0 = time.perf_counter()
    _, used = O.sweep_parallel(O.BCC, CPU_SAMPLE_DIMS, WORK.M, WORK.K, V, sig, T_KELVIN, n_sweeps, SEED,
                               L=CPU_SAMPLE_SCHED[0], nt=CPU_SAMPLE_SCHED[1], threads=os.cpu_count() or 1,
                               proposal=PROPOSAL)
    dt = time.perf_counter() - t0
    n = sig.size * n_sweeps
    t1 = time.perf_counter()
    O.sweep(O.BCC, CPU_SAMPLE_DIMS, WORK.M, WORK.K, V, sig, T_KELVIN, n_serial, SEED, sweep0=n_sweeps,
            L=CPU_SAMPLE_SCHED[0], nt=CPU_SAMPLE_SCHED[1], proposal=PROPOSAL)
    dts = time.perf_counter() - t1
    return {"value": n / dt, "unit": UNIT, "cores": used, "kind": "oracle",
            "serial_value": sig.size * n_serial / dts,
            "sample": f"C oracle, OpenMP over the sites of each phase ({used} threads), BCC "
                      f"{CPU_SAMPLE_DIMS[0]}^3 ({sig.size} sites), 4 species, 4 shells, {T_KELVIN:.0f} K, "
                      f"shared-direction proposals, "
                      f"schedule L={CPU_SAMPLE_SCHED[0]} tiles {CPU_SAMPLE_SCHED[1]}, {n_sweeps} sweeps = {n} "
                      f"trials in {dt:.1f} s; serial_value: the same oracle on 1 core, {n_serial} sweeps"}


def config_block(extra=None):
    c = {"workload": f"BCC {WORK.dims[0]}^3 cells x 2 = {WORK.sites:,} sites, 4 species equiatomic, "
                     f"packed 4-bit, 4-shell int32 EPI N(0,{WORK.sigma_mev:.0f} meV), {T_KELVIN:.0f} K",
         "sites": WORK.sites, "lattice": "bcc", "dims": list(WORK.dims), "species": WORK.M, "shells": WORK.K,
         "storage": "packed4", "temperature_K": T_KELVIN, "step": "one sweep (one swap trial per site)",
         "l2": "inputs larger than L2 (512 MB lattice store vs 129 MB L2)",
         "proposal": "shared direction: one shell-1 direction per (sweep, tile, intra colour); acceptance "
                     "uniforms per trial"}
    if extra:
        c.update(extra)
    return c


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle (OpenMP over the sites of each phase, all
    host cores), each step one sweep of a BCC 64^3 sample of the workload."""
    if rank != 0:
        return
    import oracle as O

    V = epi_gaussian(WORK.K, WORK.M, WORK.sigma_mev, WORK.epi_seed)
    sig = O.init_config(O.BCC, CPU_SAMPLE_DIMS, WORK.M, equiatomic(WORK.M), WORK.init_seed)
    sw = 0
    threads = os.cpu_count() or 1
    used = 1
    for _ in range(args.warmup):
        _, used = O.sweep_parallel(O.BCC, CPU_SAMPLE_DIMS, WORK.M, WORK.K, V, sig, T_KELVIN, 1, SEED, sweep0=sw,
                                   L=CPU_SAMPLE_SCHED[0], nt=CPU_SAMPLE_SCHED[1], threads=threads,
                                   proposal=PROPOSAL)
        sw += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, used = O.sweep_parallel(O.BCC, CPU_SAMPLE_DIMS, WORK.M, WORK.K, V, sig, T_KELVIN, 1, SEED, sweep0=sw,
                                   L=CPU_SAMPLE_SCHED[0], nt=CPU_SAMPLE_SCHED[1], threads=threads,
                                   proposal=PROPOSAL)
        sw += 1
    dt = time.perf_counter() - t0
    val = sig.size * args.steps / dt
    sample = (f"C oracle, OpenMP over the sites of each phase ({used} threads), one sweep of BCC "
              f"{CPU_SAMPLE_DIMS[0]}^3 ({sig.size} sites) per step, same species/shells/temperature/"
              f"schedule shape/proposal mode")
    out = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
           "config": config_block({"sample": sample}), "impl": "reference",
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


BATCH_R, BATCH_SWEEPS = 64, 500


def run_batched(stream):
    """64 BCC replicas with cubic edges drawn from 24..96, temperatures
    log-spaced 300-3000 K, shared 4-shell EPI: 500 sweeps in one persistent
    launch (graph-replayed, autotuned schedules), with shared-direction
    proposals (the headline's mode) and with per-trial directions.  Per-trial
    directions are also run as 64 separate handles, one smcx_sweep call each;
    both from the same start, compared bit for bit at the end.  The
    shared-direction batch is compared bit for bit with plain runs of 2
    sweeps."""
    import torch
    from paper_2503_12591_gb300 import smcx

    edges = batched_edges(BATCH_R, 24, 96, 1)
    T = log_temperatures(BATCH_R, 300.0, 3000.0)
    V = epi_gaussian(4, 4, 20.0, 1)

    def make(r, mode):
        n = int(edges[r])
        lat = smcx.Lattice(smcx.BCC, (n, n, n), 4, equiatomic(4), init_seed=1000 + r, storage=smcx.INT8,
                           stream=stream)
        lat.set_replica(r)
        lat.set_epi(V)
        lat.set_proposal(mode)
        return lat

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    def one_mode(mode, plain_sweeps):
        lats = [make(r, mode) for r in range(BATCH_R)]
        b = smcx.Batch(lats, stream)
        threads = b.autotune(T, trial_sweeps=8)  # near-equal candidates: enough sweeps to rank them
        scheds = [l.schedule() for l in lats]
        plain = [make(r, mode) for r in range(BATCH_R)]
        for p, sc in zip(plain, scheds):
            p.set_schedule(sc)
            if mode == smcx.PROPOSAL_SITE:
                p.set_block(threads)
        b.sweep(T, 2, SEED)
        for r, p in enumerate(plain):
            p.sweep(T[r], 2, SEED)

        def same():
            return all((l.get_config() == p.get_config()).all() and
                       l.state()[1].tolist() == p.state()[1].tolist() for l, p in zip(lats, plain))

        exact = same() if not plain_sweeps else None
        ms_b = timed(lambda: b.sweep(T, BATCH_SWEEPS, SEED))
        info = b.info()
        ms_p = None
        if plain_sweeps:
            ms_p = timed(lambda: [p.sweep(T[r], plain_sweeps, SEED) for r, p in enumerate(plain)])
            exact = same()
        b.close()
        for l in lats + plain:
            l.close()
        return ms_b, ms_p, info, exact, scheds

    sites = sum(2 * int(n) ** 3 for n in edges)
    att = sites * BATCH_SWEEPS
    ms_d, _, info_d, exact_d, sch_d = one_mode(smcx.PROPOSAL_TILE, 0)
    ms_b, ms_p, info, exact, _ = one_mode(smcx.PROPOSAL_SITE, BATCH_SWEEPS)
    return {"value": att / (ms_d / 1e3), "unit": UNIT, "proposal": "shared direction per (sweep, tile, phase)",
            "replicas": BATCH_R, "sites": sites, "sweeps": BATCH_SWEEPS, "ms_batched": ms_d, "graph": info_d["graph"],
            "grid": info_d["grid"], "threads": info_d["threads"], "schedule_L": sch_d[0][0],
            "bit_exact_vs_plain": bool(exact_d),
            "per_trial_direction": {"value": att / (ms_b / 1e3), "ms_batched": ms_b, "grid": info["grid"],
                                    "threads": info["threads"], "plain_value": att / (ms_p / 1e3),
                                    "speedup_vs_plain": ms_p / ms_b, "ms_plain": ms_p,
                                    "bit_exact_vs_plain": bool(exact),
                                    "plain": "64 handles, one smcx_sweep call each (8 tile-colour launches per sweep)"},
            "workload": "64 BCC cubic lattices, edges U{24..96} (seed 1), 4 species, shared 4-shell EPI, "
                        "T log-spaced 300-3000 K, int8 storage"}


EX_R, EX_EDGE, EX_ROUNDS, EX_SPR = 32, 48, 40, 10


def run_batch_launch(stream, proposal, sched):
    """Profiling aid: the 64-replica batched workload with a fixed schedule
    (link cell L, tiles of at most `target` cells, `threads` per CTA), one
    warm-up launch and one more launch of one sweep each, so that a profiler
    can capture the second launch alone."""
    import torch
    from paper_2503_12591_gb300 import smcx

    L, target, threads = (int(x) for x in sched.split(","))
    edges = batched_edges(BATCH_R, 24, 96, 1)
    T = log_temperatures(BATCH_R, 300.0, 3000.0)
    V = epi_gaussian(4, 4, 20.0, 1)
    lats = []
    for r in range(BATCH_R):
        n = int(edges[r])
        lat = smcx.Lattice(smcx.BCC, (n, n, n), 4, equiatomic(4), init_seed=1000 + r, storage=smcx.INT8,
                           stream=stream)
        lat.set_replica(r)
        lat.set_epi(V)
        lat.set_proposal(proposal)
        nt = 2
        while (n + nt - 1) // nt > target:
            nt += 2
        lat.set_schedule((L, (nt, nt, nt)))
        lats.append(lat)
    b = smcx.Batch(lats, stream)
    b.set_block(threads)
    b.sweep(T, 1, SEED)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.sweep(T, 1, SEED)
    e1.record(stream)
    e1.synchronize()
    info = b.info()
    b.close()
    for l in lats:
        l.close()
    return {"proposal": proposal, "schedule": [L, target, threads], "ms_launch": e0.elapsed_time(e1),
            "grid": info["grid"], "threads": info["threads"], "sites": sum(2 * int(n) ** 3 for n in edges)}


def run_qsro_launch(stream, edge=0):
    """Profiling aid: the qSRO workload (FCC 400^3 unless --edge) with the
    schedule of its bench line fixed (link cells of 4, 20 tiles per axis),
    one warm-up sweep and one more sweep, so that a profiler can capture a
    launch of the second sweep alone (skip the first sweep's 8)."""
    import torch
    from paper_2503_12591_gb300 import smcx
    from paper_2503_12591_gb300.inputs import SCALE_FCC400 as W_

    if edge:
        import dataclasses
        W_ = dataclasses.replace(W_, dims=(edge,) * 3)
    W = np.random.default_rng(77).integers(-300, 301, (W_.K, W_.M)).astype(np.int32)
    lat = smcx.Lattice(W_.kind, W_.dims, W_.M, W_.comp, init_seed=W_.init_seed, storage=W_.storage, stream=stream)
    lat.set_epi(W_.epi())
    lat.set_qsro(W)
    nt = 2
    while -(-W_.dims[0] // nt) > 20:
        nt += 2
    lat.set_schedule((4, (nt, nt, nt)))
    lat.sweep(1000.0, 1, SEED)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.sweep(1000.0, 1, SEED)
    e1.record(stream)
    e1.synchronize()
    lat.close()
    return {"edge": W_.dims[0], "schedule": [4, nt], "ms_sweep": e0.elapsed_time(e1)}


def run_exchange(stream):
    """Replica exchange: 32 BCC 48^3 replicas (221,184 sites each) on
    temperature slots 600-1400 K (linear), 40 rounds of 10 batched sweeps +
    one exchange step, against the same 400 batched sweeps with no exchange."""
    import time as _t

    import torch
    from paper_2503_12591_gb300 import smcx

    V = epi_gaussian(4, 4, 20.0, 1)
    T_slot = np.linspace(600.0, 1400.0, EX_R)

    def make(r):
        lat = smcx.Lattice(smcx.BCC, (EX_EDGE,) * 3, 4, equiatomic(4), init_seed=2000 + r, storage=smcx.INT8,
                           stream=stream)
        lat.set_replica(r)
        lat.set_epi(V)
        return lat

    lats = [make(r) for r in range(EX_R)]
    sites = sum(l.N for l in lats)
    b = smcx.Batch(lats, stream)
    rep, ctr, acc = b.exchange(T_slot, np.arange(EX_R), 2, EX_SPR, SEED)  # warm-up, graph capture
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    rep, ctr, acc = b.exchange(T_slot, rep, EX_ROUNDS, EX_SPR, SEED, round_ctr=ctr, accepts=acc)
    torch.cuda.synchronize()
    s_ex = _t.perf_counter() - t0
    T_rep = np.empty(EX_R)
    T_rep[rep] = T_slot
    b.sweep(T_rep, EX_SPR, SEED)
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    for _ in range(EX_ROUNDS):
        b.sweep(T_rep, EX_SPR, SEED)
    torch.cuda.synchronize()
    s_plain = _t.perf_counter() - t0
    b.close()
    for l in lats:
        l.close()
    att = sites * EX_ROUNDS * EX_SPR
    n_prop = sum(len(range(i & 1, EX_R - 1, 2)) for i in range(ctr))  # proposals since the first exchange round
    return {"value": att / s_ex, "unit": UNIT, "no_exchange_value": att / s_plain, "overhead": s_ex / s_plain,
            "exchange_acceptance": float(acc.sum()) / max(1, n_prop),
            "replicas": EX_R, "sites": sites, "rounds": EX_ROUNDS, "sweeps_per_round": EX_SPR,
            "workload": f"{EX_R} x BCC {EX_EDGE}^3 int8, shared 4-shell EPI, T slots 600-1400 K linear; "
                        "host wall time per round: batched sweeps + exact energies + exchange step"}


def run_throughput256(stream):
    """The 33.5M-site throughput workload: BCC 256^3 int8, 1000 sweeps at each
    of 2500, 1500 and 800 K, energy + Warren-Cowley SRO every 100 sweeps;
    timed with CUDA events with and without the observables (the 33.5 MB
    lattice fits the 129 MB L2, so this runs from L2, not HBM)."""
    import torch
    from paper_2503_12591_gb300 import smcx
    from paper_2503_12591_gb300.inputs import THROUGHPUT_BCC256 as W_

    lat = smcx.Lattice(W_.kind, W_.dims, W_.M, W_.comp, init_seed=W_.init_seed, storage=W_.storage, stream=stream)
    lat.set_epi(W_.epi())
    default_sched = lat.schedule()
    (L, nt), th = lat.autotune(W_.temperatures[1], 2)  # outside the timed region; state restored
    lat.sweep(W_.temperatures[0], 3, SEED)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per_T = []
    t_all = 0.0
    n_sw = 0
    for T in W_.temperatures:
        e0.record(stream)
        obs = []
        for _ in range(10):
            lat.sweep(T, 100, SEED)
            obs.append((lat.energy(), lat.sro()[0, 0, 1]))
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        t_all += ms
        n_sw += 1000
        per_T.append({"T": T, "ms_1000_sweeps_with_observables": ms,
                      "final_energy": int(obs[-1][0]), "final_alpha1_01": float(obs[-1][1])})
    e0.record(stream)
    lat.sweep(W_.temperatures[-1], 200, SEED)
    e1.record(stream)
    e1.synchronize()
    ms_plain = e0.elapsed_time(e1) / 200
    N = lat.N
    lat.close()
    return {"value": N * n_sw / (t_all / 1e3), "unit": UNIT, "sweep_only_value": N / (ms_plain / 1e3),
            "per_temperature": per_T,
            "schedule": {"L": L, "tiles": list(nt), "threads": th, "autotuned": True,
                         "default": {"L": default_sched[0], "tiles": list(default_sched[1])}},
            "workload": "BCC 256^3 = 33,554,432 sites int8, 4 species, 4-shell EPI N(0,20 meV); 1000 sweeps at "
                        "2500/1500/800 K, E + SRO every 100 sweeps (value includes them); L2-resident"}


def run_fcc(stream, edge=0):
    """The FCC scale workload (400^3 = 256M sites, 5 species, 3 shells, packed
    4-bit, 1200 K; the paper's FeCoNiAlTi-like system): pair-model sweeps on
    the FCC tile kernel with shared-direction proposals (the headline's mode),
    with the library's schedule and then the autotuned one; and with a
    direction drawn per trial."""
    import torch
    from paper_2503_12591_gb300 import smcx
    from paper_2503_12591_gb300.inputs import SCALE_FCC400 as W_

    if edge:
        import dataclasses
        W_ = dataclasses.replace(W_, dims=(edge,) * 3)
    lat = smcx.Lattice(W_.kind, W_.dims, W_.M, W_.comp, init_seed=W_.init_seed, storage=W_.storage, stream=stream)
    lat.set_epi(W_.epi())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    T = W_.temperatures[0]

    def timed(n):
        lat.sweep(T, 2, SEED)
        torch.cuda.synchronize()
        e0.record(stream)
        lat.sweep(T, n, SEED)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / n

    sched = lat.schedule()
    lat.set_proposal(smcx.PROPOSAL_TILE)
    ms = timed(10)
    (L, nt), _ = lat.autotune(T, 2)
    ms_t = timed(10)
    lat.set_proposal(smcx.PROPOSAL_SITE)
    ms_site = timed(10)
    N = lat.N
    lat.close()
    return {"value": N / (ms / 1e3), "unit": UNIT, "ms_per_sweep": ms,
            "proposal": "shared direction per (sweep, tile, intra colour)",
            "schedule": {"L": sched[0], "tiles": list(sched[1])},
            "autotuned_value": N / (ms_t / 1e3), "autotuned_schedule": {"L": L, "tiles": list(nt)},
            "per_trial_direction_value": N / (ms_site / 1e3),
            "kernel": "k_fcc_tile_sweep<3,0,0,1> (per-trial: <3,0,0,0>)",
            "workload": f"FCC {W_.dims[0]}^3 = {N:,} sites, 5 species 0.3/0.25/0.2/0.15/0.1, 3-shell EPI "
                        "N(0,30 meV), packed 4-bit, 1200 K"}


def run_qsro(stream, edge=0):
    """qSRO model (pair terms + W_k[s_i] n_k(i)^2) on the FCC 400^3 scale
    workload (256M sites, 5 species, packed 4-bit, 3 shells), W ~ U{-300..300}
    (0.01 meV, seed 77), 1000 K, sweeps timed with
    CUDA events, against the pair model on the same lattice; both schedules
    autotuned (smcx_autotune) outside the timed region."""
    import torch
    from paper_2503_12591_gb300 import smcx
    from paper_2503_12591_gb300.inputs import SCALE_FCC400 as W_

    if edge:
        import dataclasses
        W_ = dataclasses.replace(W_, dims=(edge,) * 3)
    W = np.random.default_rng(77).integers(-300, 301, (W_.K, W_.M)).astype(np.int32)
    lat = smcx.Lattice(W_.kind, W_.dims, W_.M, W_.comp, init_seed=W_.init_seed, storage=W_.storage, stream=stream)
    lat.set_epi(W_.epi())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(n):
        lat.sweep(1000.0, 1, SEED)
        torch.cuda.synchronize()
        e0.record(stream)
        lat.sweep(1000.0, n, SEED)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / n

    lat.autotune(1000.0, 1)
    ms_pair = timed(3)
    sched_pair = lat.schedule()
    lat.set_schedule(None)  # the tuned pair schedule is too small for the qSRO reach
    lat.set_qsro(W)
    lat.autotune(1000.0, 1)
    ms_q = timed(2)
    sched_q = lat.schedule()
    st = lat.state()[1]
    lat.close()
    N = W_.sites
    return {"value": N / (ms_q / 1e3), "unit": UNIT, "ms_per_sweep": ms_q,
            "pair_model_value": N / (ms_pair / 1e3), "slowdown_vs_pair": ms_q / ms_pair,
            "schedule": {"L": sched_q[0], "tiles": list(sched_q[1])},
            "pair_schedule": {"L": sched_pair[0], "tiles": list(sched_pair[1])},
            "acceptance": float(st[1]) / max(1, int(st[0])),
            "kernel": "k_qsro_fcc_n<3>" if max(-(-d // t) for d, t in zip(W_.dims, sched_q[1])) <= 20
                      else "k_tile_sweep_qsro<FCC,3>",
            "workload": f"FCC {W_.dims[0]}^3 = {N / 1e6:.0f}M sites, 5 species 0.3/0.25/0.2/0.15/0.1, 3-shell EPI "
                        "N(0,30 meV) + qSRO W U{-300..300} (0.01 meV), packed 4-bit, 1000 K"}


# The five runs of the paper's Tab. models_summary (H800; sweep times as
# printed there): name, lattice, cells, species composition, energy model, T_sweep (s).
FECONIALTI = [0.29, 0.29, 0.28, 0.07, 0.07]   # Fe29Co29Ni28Al7Ti7 (Results, FeCoNiAlTi section)
PAPER_ROWS = [
    ("MoNbTaW_1B_EPI", "bcc", (795, 795, 795), [0.25] * 4, "epi", 0.1912),
    ("FeCoNiAlTi_1B_EPI", "fcc", (630, 630, 630), FECONIALTI, "epi", 0.4120),
    ("FeCoNiAlTi_1B_qSRO", "fcc", (632, 632, 632), FECONIALTI, "qsro", 21.65),
    ("FeCoNiAlTi_1M_EPI", "fcc", (72, 60, 60), FECONIALTI, "epi", 0.001755),
    ("FeCoNiAlTi_1M_qSRO", "fcc", (72, 60, 60), FECONIALTI, "qsro", 0.04703),
]


def run_paper_rows(stream):
    """The shapes of the paper's five timed runs (Tab. models_summary): same
    lattices, cell counts, species counts and 2-shell (2NN) models, with
    synthetic seeded tables in place of the unpublished trained ones (EPI
    N(0, 20 meV) BCC / N(0, 30 meV) FCC, qSRO W ~ U{-300..300} 0.01 meV),
    packed 4-bit, 1000 K.  Sweeps timed with CUDA events after a warm-up;
    schedules autotuned outside the timed region except for the 1B qSRO run
    (library schedule: 4-cell link cells as in the paper, 20-cell tiles).  The
    paper's figures are another GPU (H800) and other tables: context, not
    the target."""
    import torch
    from paper_2503_12591_gb300 import smcx

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    for name, kind, dims, comp, model, t_paper in PAPER_ROWS:
        M, K = len(comp), 2
        lat = smcx.Lattice(smcx.BCC if kind == "bcc" else smcx.FCC, dims, M, comp, init_seed=11,
                           storage=smcx.PACKED4, stream=stream)
        lat.set_epi(epi_gaussian(K, M, 20.0 if kind == "bcc" else 30.0, 5))
        if model == "qsro":
            lat.set_qsro(np.random.default_rng(77).integers(-300, 301, (K, M)).astype(np.int32))
        big = lat.N > 10**8
        if not (big and model == "qsro"):
            lat.autotune(1000.0, 1 if big else 5)
        n = 2 if model == "qsro" and big else 5 if big else 50 if model == "qsro" else 200
        lat.sweep(1000.0, 1, SEED)
        torch.cuda.synchronize()
        e0.record(stream)
        lat.sweep(1000.0, n, SEED)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / n
        L, nt = lat.schedule()
        N = lat.N
        lat.close()
        rows.append({"name": name, "sites": N, "model": f"{model} 2 shells", "species": M,
                     "value": N / (ms / 1e3), "ms_per_sweep": ms, "sweeps_timed": n,
                     "schedule": {"L": L, "tiles": list(nt)},
                     "paper_T_sweep_s": t_paper, "paper_value": N / t_paper,
                     "ratio_vs_paper": (N / (ms / 1e3)) / (N / t_paper)})
    return {"unit": UNIT, "rows": rows,
            "note": "the paper's Tab. models_summary shapes with synthetic 2-shell tables at 1000 K; the paper's "
                    "sweep times are on an H800 with its trained tables (context, not vs_baseline)"}


def run_anneal(stream):
    """The annealing driver on BCC 320^3 (65.5M sites, packed, the workload's
    4-species 4-shell EPI): 2000 K down to 1000 K in 50 K steps (the paper's
    schedule), 20 sweeps discarded and 40 recorded per temperature, exact
    energy after every recorded sweep, C_V per site from its variance.  (A
    checkerboard sweep runs (n / 2L)^3 trials at a time whatever the tiling,
    so lattices much smaller than this leave the GPU idle: 4,096 at 128^3.)"""
    import time as _t

    import torch
    from paper_2503_12591_gb300 import anneal, smcx

    lat = smcx.Lattice(smcx.BCC, (320, 320, 320), WORK.M, WORK.comp, init_seed=3, storage=smcx.PACKED4,
                       stream=stream)
    lat.set_epi(WORK.epi())
    temps = anneal.paper_schedule()
    lat.sweep(temps[0], 2, SEED)
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    steps = anneal.anneal(lat, temps, discard=20, record=40, seed=SEED)
    dt = _t.perf_counter() - t0
    n_sw = len(temps) * 60
    N = lat.N
    lat.close()
    cv = [s.cv_per_site for s in steps]
    k = int(np.argmax(cv))
    return {"value": N * n_sw / dt, "unit": UNIT, "seconds": dt, "sweeps": n_sw, "temperatures": len(temps),
            "cv_per_site_max": cv[k], "cv_peak_T": steps[k].T,
            "cv_per_site": [round(c, 4) for c in cv], "acceptance_last_T": steps[-1].accept_rate,
            "note": "a throughput measurement of the driver: 20 + 40 sweeps per temperature are far too few for "
                    "equilibrium (the paper discards 4e5-1.5e6 sweeps per temperature), so these C_V values "
                    "include the relaxation drift after each temperature step and are not physical",
            "workload": "BCC 320^3 = 65,536,000 sites packed 4-bit, 4 species, 4-shell EPI N(0,20 meV); "
                        "2000 -> 1000 K in 50 K steps, 20 discarded + 40 recorded sweeps per temperature; "
                        "host wall time including the per-sweep exact energies and their FP64 moments on the device "
                        "(smcx_sweep_cv)"}


def run_clusters(stream, edge=0):
    """Local-energy field and union-find clusters on the FCC 400^3 scale
    workload (256M sites, 5 species, packed 4-bit) after one sweep at 1200 K,
    threshold = median of a 1/97 sample of 2 E_i; CUDA events on the stream."""
    import torch
    from paper_2503_12591_gb300 import smcx
    from paper_2503_12591_gb300.inputs import SCALE_FCC400 as W

    if edge:
        import dataclasses
        W = dataclasses.replace(W, dims=(edge,) * 3)
    lat = smcx.Lattice(W.kind, W.dims, W.M, W.comp, init_seed=W.init_seed, storage=W.storage, stream=stream)
    lat.set_epi(W.epi())
    lat.sweep(W.temperatures[0], 1, W.seed)
    N = lat.N
    e2 = torch.empty(N, dtype=torch.int32, device="cuda")
    lab = torch.empty(N, dtype=torch.int32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    lat.local_energy(e2.data_ptr())  # warm-up
    lat.synchronize()
    thr = int(torch.kthvalue(e2[::97].cpu(), e2[::97].numel() // 2).values.item())
    lat.clusters(thr, lab.data_ptr())
    torch.cuda.synchronize()
    ev[0].record(stream)
    lat.local_energy(e2.data_ptr())
    ev[1].record(stream)
    nc = lat.clusters(thr, lab.data_ptr())
    ev[2].record(stream)
    roots, sizes, _ = lat.cluster_summary(lab.data_ptr(), 100, 16)
    ev[3].record(stream)
    ev[3].synchronize()
    ms_e, ms_c, ms_s = (ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3]))
    lat.close()
    return {"sites": N, "ms_local_energy": ms_e, "ms_clusters": ms_c, "ms_summary": ms_s,
            "local_energy_sites_per_s": N / (ms_e / 1e3), "clusters_sites_per_s": N / (ms_c / 1e3),
            "n_clusters": nc, "largest": [int(x) for x in sizes[:5]],
            "workload": "FCC 400^3 = 256M sites, 5 species 0.3/0.25/0.2/0.15/0.1, 3-shell EPI N(0,30 meV), "
                        "packed 4-bit, one sweep at 1200 K; class = 2E_i < median; shell-1 connectivity; "
                        "clusters = local energies + union-find + compression; summary >= 100 sites"}


def run_gradient(stream):
    """Differentiation workloads.  (a) EPI fit: 4096 equiatomic BCC 8^3
    configurations (1024 sites, seed = index), hidden 4-shell EPI N(0,20 meV)
    (seed 7), FP32 per-site targets + N(0,1 meV) noise; pair counts batched
    vs one configuration per launch, then forward + backward + Adam steps.
    (b) Fluctuation gradient d<alpha_1>/dV: 64 replicas of BCC 48^3 at
    1000 K, 2000 sweeps (500 burn-in), FP64 accumulation after every sweep,
    against the same sweeps without accumulation."""
    import torch
    from paper_2503_12591_gb300 import diff, smcx

    dev = torch.device("cuda")
    out = {}
    # (a) fitting step
    B, dims, M, K = 4096, (8, 8, 8), 4, 4
    N = 2 * 8 ** 3
    rng_cfg = [np.random.default_rng(b).permutation(np.repeat(np.arange(M), N // M)) for b in range(B)]
    cfg = torch.from_numpy(np.stack(rng_cfg).astype(np.int8)).to(dev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    C = diff.pair_counts(cfg, smcx.BCC, dims, M, K)
    e0.record(stream)
    C = diff.pair_counts(cfg, smcx.BCC, dims, M, K)
    e1.record(stream)
    e1.synchronize()
    ms_batched = e0.elapsed_time(e1)
    Cp = torch.empty_like(C)
    e0.record(stream)
    for b in range(B):
        smcx.pair_counts_batch(smcx.BCC, dims, M, K, cfg[b].data_ptr(), 1, Cp[b].data_ptr(), stream.cuda_stream)
    e1.record(stream)
    e1.synchronize()
    ms_plain = e0.elapsed_time(e1)
    exact = bool(torch.equal(C, Cp))
    Vh = torch.tensor(epi_gaussian(K, M, 20.0, 7), dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev).manual_seed(7)
    with torch.no_grad():
        target = diff.epi_energy(Vh, C) / N / 100.0 + torch.randn(B, device=dev, generator=gen)
    W = torch.zeros((K, M, M), device=dev, requires_grad=True)
    opt = torch.optim.Adam([W], lr=5.0)

    def step():
        opt.zero_grad(set_to_none=True)
        V = 0.5 * (W + W.transpose(1, 2))
        pred = diff.epi_energy(V * 100.0, C) / N / 100.0
        loss = torch.mean((pred - target) ** 2)
        loss.backward()
        opt.step()
        return loss

    for _ in range(3):
        step()
    n_steps = 50
    e0.record(stream)
    for _ in range(n_steps):
        loss = step()
    e1.record(stream)
    e1.synchronize()
    ms_fit = e0.elapsed_time(e1) / n_steps
    out["fit"] = {"configs_per_s_pair_counts_batched": B / (ms_batched / 1e3),
                  "configs_per_s_pair_counts_plain": B / (ms_plain / 1e3),
                  "speedup_vs_plain": ms_plain / ms_batched, "bit_exact_vs_plain": exact,
                  "fit_step_ms": ms_fit, "fit_configs_per_s": B / (ms_fit / 1e3),
                  "final_loss_meV2": float(loss.item()),
                  "plain": "one configuration per smcx_pair_counts_batch launch",
                  "workload": "4096 BCC 8^3 configs x 1024 sites, 4 species, 4-shell EPI fit (Adam)"}
    # (b) fluctuation gradient
    R, n, T, burn, total = 64, 48, 1000.0, 500, 2000
    V = epi_gaussian(4, 4, 20.0, 1)

    def make_set():
        lats = []
        for r in range(R):
            l = smcx.Lattice(smcx.BCC, (n, n, n), 4, equiatomic(4), init_seed=500 + r, storage=smcx.INT8,
                             stream=stream)
            l.set_replica(r)
            l.set_epi(V)
            lats.append(l)
        return lats

    Ts = [T] * R
    lats = make_set()
    b = smcx.Batch(lats, stream)
    b.sweep(Ts, burn, SEED)
    est = diff.BatchFluctuationEstimator(b, 4, 4, 0)  # every replica in two launches per sample
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(total - burn):
        b.sweep(Ts, 1, SEED)
        est.add()
    torch.cuda.synchronize()
    s_acc = time.perf_counter() - t0
    grads = est.gradients(T)
    g_mean = grads.mean(0)
    g_se = grads.std(0) / np.sqrt(R)
    b.close()
    lats2 = make_set()
    b2 = smcx.Batch(lats2, stream)
    b2.sweep(Ts, burn, SEED)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(total - burn):
        b2.sweep(Ts, 1, SEED)
    torch.cuda.synchronize()
    s_plain = time.perf_counter() - t0
    same = all((l.get_config() == l2.get_config()).all() for l, l2 in zip(lats, lats2))
    b2.close()
    for l in lats + lats2:
        l.close()
    k01 = g_mean[1, 0, 0, 1].item() + g_mean[1, 0, 1, 0].item()
    out["fluctuation"] = {"sweeps_per_s_with_accumulation": (total - burn) / s_acc,
                          "sweeps_per_s_without": (total - burn) / s_plain,
                          "overhead": s_acc / s_plain,
                          "configs_identical_with_and_without": bool(same),
                          "dalpha1_AB_dV1_AB_per_meV": k01,
                          "max_rel_stderr": float((g_se.abs() / g_mean.abs().clamp_min(1e-12)).median()),
                          "workload": "64 x BCC 48^3, 1000 K, 2000 sweeps (500 burn-in), d<alpha_1>/dV FP64, "
                                      "measured after every sweep; batched sweeps one call per sweep; sums of all replicas by smcx_batch_fluct_accumulate (two launches)"}
    return out


def run_baselines(stream):
    """Per-config oracle timings (the C oracle as it stands, serial and OpenMP
    on all host cores) on bounded samples, and the GPU time of the
    oracle-sized config 1 (BCC 16^3, 100 sweeps).  Samples that are smaller
    than their config are labelled with what was timed; a rate measured on a
    sample stands for the config's per-trial rate (the oracle's cost per trial
    does not depend on the lattice size)."""
    import torch

    import oracle as O
    from paper_2503_12591_gb300 import smcx
    from paper_2503_12591_gb300.inputs import ORACLE_BCC16, SCALE_FCC400, THROUGHPUT_BCC256

    cores = os.cpu_count() or 1
    out = {"cores": cores}

    def oracle_rate(kind, dims, M, comp, K, V, T, n_sweeps, sched, proposal=0, threads=1, init_seed=1):
        sig = O.init_config(kind, dims, M, comp, init_seed)
        t0 = time.perf_counter()
        if threads == 1:
            O.sweep(kind, dims, M, K, V, sig, T, n_sweeps, SEED, L=sched[0], nt=sched[1], proposal=proposal)
            used = 1
        else:
            _, used = O.sweep_parallel(kind, dims, M, K, V, sig, T, n_sweeps, SEED, L=sched[0], nt=sched[1],
                                       threads=threads, proposal=proposal)
        dt = time.perf_counter() - t0
        return sig.size * n_sweeps / dt, used, dt

    # config 1: BCC 16^3 int8, 100 sweeps at 1000 K, in full (GPU and oracle)
    w = ORACLE_BCC16
    V1 = w.epi()
    lat = smcx.Lattice(w.kind, w.dims, w.M, w.comp, init_seed=w.init_seed, storage=smcx.INT8, stream=stream)
    lat.set_epi(V1)
    sched1 = lat.schedule()
    lat.sweep(w.temperatures[0], 3, w.seed)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.sweep(w.temperatures[0], w.sweeps, w.seed)
    e1.record(stream)
    e1.synchronize()
    ms1 = e0.elapsed_time(e1)
    lat.close()
    r1s, _, _ = oracle_rate(w.kind, w.dims, w.M, w.comp, w.K, V1, w.temperatures[0], w.sweeps, sched1)
    r1p, used, _ = oracle_rate(w.kind, w.dims, w.M, w.comp, w.K, V1, w.temperatures[0], w.sweeps, sched1,
                               threads=cores)
    out["config1"] = {"gpu": w.sites * w.sweeps / (ms1 / 1e3), "gpu_ms_100_sweeps": ms1,
                      "oracle_1core": r1s, "oracle_cores": r1p, "oracle_threads": used,
                      "schedule": {"L": sched1[0], "tiles": list(sched1[1])},
                      "sample": "in full: 8192 sites x 100 sweeps (GPU and oracle)"}
    # config 2: BCC 256^3 int8 at 2500 K: oracle on 1 sweep (OpenMP) / 1 sweep of BCC 64^3 (serial)
    w = THROUGHPUT_BCC256
    V2 = w.epi()
    s2 = (3, (18, 18, 18))
    r2p, used, dt2 = oracle_rate(w.kind, w.dims, w.M, w.comp, w.K, V2, w.temperatures[0], 1, s2, threads=cores)
    r2s, _, _ = oracle_rate(w.kind, (64, 64, 64), w.M, w.comp, w.K, V2, w.temperatures[0], 1, (3, (4, 4, 4)))
    out["config2"] = {"oracle_cores": r2p, "oracle_threads": used, "oracle_1core": r2s,
                      "sample": f"OpenMP: one sweep of the full 33.5M-site lattice ({dt2:.1f} s); 1 core: one "
                                "sweep of BCC 64^3 (same model and temperature)"}
    # config 3a: BCC 800^3 packed, shared-direction proposals: oracle rate on BCC 128^3 (1 sweep)
    r3p, used, _ = oracle_rate(smcx.BCC, (128, 128, 128), WORK.M, WORK.comp, WORK.K, WORK.epi(), T_KELVIN, 1,
                               (4, (16, 16, 16)), proposal=PROPOSAL, threads=cores)
    r3s, _, _ = oracle_rate(smcx.BCC, (64, 64, 64), WORK.M, WORK.comp, WORK.K, WORK.epi(), T_KELVIN, 1,
                            (4, (8, 8, 8)), proposal=PROPOSAL)
    out["config3a"] = {"oracle_cores": r3p, "oracle_threads": used, "oracle_1core": r3s,
                       "sample": "OpenMP: one sweep of BCC 128^3 (4.2M sites); 1 core: one sweep of BCC 64^3; "
                                 "same model, temperature and proposal mode as the 800^3 workload"}
    # config 3a in full: one sweep of the 1.024B-site lattice by the oracle (OpenMP) and by the GPU, from
    # the same seeded equiatomic start (numpy), in the bench's schedule and proposal mode; compared bit for
    # bit (configuration and statistics)
    n_full = 2 * 800 ** 3
    start = np.repeat(np.arange(WORK.M, dtype=np.int8), n_full // WORK.M)
    np.random.default_rng(2024).shuffle(start)
    lat = smcx.Lattice(smcx.BCC, (800, 800, 800), WORK.M, WORK.comp, init_seed=1, storage=smcx.PACKED4,
                       sched=(4, (40, 40, 40)), stream=stream)
    lat.set_config(start)
    lat.set_epi(WORK.epi())
    lat.set_proposal(PROPOSAL)
    lat.sweep(T_KELVIN, 1, SEED)
    got = lat.get_config()
    st_gpu = lat.state()[1]
    lat.close()
    sig = start
    del start
    t0 = time.perf_counter()
    st_orc, used = O.sweep_parallel(smcx.BCC, (800, 800, 800), WORK.M, WORK.K, WORK.epi(), sig, T_KELVIN, 1, SEED,
                                    L=4, nt=(40, 40, 40), threads=cores, proposal=PROPOSAL)
    dtf = time.perf_counter() - t0
    out["config3a_full"] = {"oracle_cores": n_full / dtf, "oracle_threads": used, "seconds": dtf,
                            "bit_exact_vs_gpu": bool((got == sig).all()) and st_orc.tolist() == st_gpu.tolist(),
                            "sample": "in full: one sweep of the 1,024,000,000-site lattice (schedule L = 4, "
                                      "40 tiles per axis, shared-direction proposals, 1200 K) from a seeded "
                                      "equiatomic numpy start, the GPU's sweep from the same start compared "
                                      "site by site"}
    del got, sig
    # config 3b: FCC 400^3 5 species: oracle rate on FCC 64^3 (1 sweep)
    w = SCALE_FCC400
    V3 = w.epi()
    r3bp, used, _ = oracle_rate(w.kind, (64, 64, 64), w.M, w.comp, w.K, V3, w.temperatures[0], 1, (3, (4, 4, 4)),
                                threads=cores)
    r3bs, _, _ = oracle_rate(w.kind, (32, 32, 32), w.M, w.comp, w.K, V3, w.temperatures[0], 1, (3, (2, 2, 2)))
    out["config3b"] = {"oracle_cores": r3bp, "oracle_threads": used, "oracle_1core": r3bs,
                       "sample": "OpenMP: one sweep of FCC 64^3 (1.05M sites); 1 core: one sweep of FCC 32^3"}
    # config 4: 64 batched replicas (edges 24..96): every replica once, 1 sweep each
    edges = batched_edges(BATCH_R)
    Vb = epi_gaussian(4, 4, 20.0, 1)
    Tb = log_temperatures(BATCH_R)
    t0 = time.perf_counter()
    nb = 0
    for r, e in enumerate(edges):
        dims = (int(e),) * 3
        sig = O.init_config(O.BCC, dims, 4, equiatomic(4), 100 + r)
        nt = 2
        while (int(e) + nt - 1) // nt > 16:
            nt += 2
        O.sweep_parallel(O.BCC, dims, 4, 4, Vb, sig, float(Tb[r]), 1, SEED, replica=r, L=3, nt=(nt,) * 3,
                         threads=cores)
        nb += sig.size
    dt4 = time.perf_counter() - t0
    out["config4"] = {"oracle_cores": nb / dt4, "oracle_threads": cores,
                      "sample": f"one sweep of each of the 64 replicas in turn ({nb:,} trials, {dt4:.1f} s, "
                                "initial placement included)"}
    # config 5a: pair counts of the 4096 BCC 8^3 configurations (the fit's forward/backward input), in full
    B, dims5, M5, K5 = 4096, (8, 8, 8), 4, 4
    N5 = 2 * 8 ** 3
    cfgs = [np.random.default_rng(b).permutation(np.repeat(np.arange(M5), N5 // M5)).astype(np.int8)
            for b in range(B)]
    t0 = time.perf_counter()
    for c in cfgs:
        O.pair_counts(O.BCC, dims5, M5, K5, c)
    dt5 = time.perf_counter() - t0
    out["config5a"] = {"oracle_1core_configs_per_s": B / dt5,
                       "sample": "pair counts of all 4096 configurations (the fit step's forward and backward "
                                 "are linear in them), serial"}
    # config 5b: fluctuation sweeps: 64 x BCC 48^3 at 1000 K, 2 sweeps + 2 pair-count samples per replica
    V5 = epi_gaussian(4, 4, 20.0, 1)
    t0 = time.perf_counter()
    n5 = 0
    for r in range(BATCH_R):
        sig = O.init_config(O.BCC, (48, 48, 48), 4, equiatomic(4), 1000 + r)
        for k in range(2):
            O.sweep_parallel(O.BCC, (48, 48, 48), 4, 4, V5, sig, 1000.0, 1, SEED, sweep0=k, replica=r, L=3,
                             nt=(4, 4, 4), threads=cores)
            O.pair_counts(O.BCC, (48, 48, 48), 4, 4, sig)
            n5 += sig.size
    dt5b = time.perf_counter() - t0
    out["config5b"] = {"oracle_cores": n5 / dt5b, "oracle_threads": cores,
                       "sample": "2 sweeps of each of the 64 BCC 48^3 replicas, each followed by its pair counts "
                                 f"(the fluctuation sample), {dt5b:.1f} s"}
    return out


def aggregate_ranks(ms, sites, steps, dist_mod=None, device="cuda"):
    """Replicas-only scaling: every rank sweeps its own lattice; the job time
    is the slowest rank's, the job's trials are the sum over ranks."""
    import torch
    world = dist_mod.get_world_size() if dist_mod is not None else 1
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if dist_mod is not None:
        dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, sites * steps * world / (ms_max / 1e3)


def run_smcx(args, rank, world, local_rank):
    import torch

    from paper_2503_12591_gb300 import smcx

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    V = WORK.epi()
    with torch.cuda.stream(stream):
        lat = smcx.Lattice(smcx.BCC, WORK.dims, WORK.M, WORK.comp, init_seed=WORK.init_seed + rank,
                           storage=smcx.PACKED4, stream=stream)
        lat.set_proposal(PROPOSAL)
        lat.set_epi(V)
    sched = lat.schedule()
    # replicas on different ranks differ by their initial configuration
    for _ in range(args.warmup):
        lat.sweep(T_KELVIN, 1, SEED)
    lat.synchronize()
    try:
        lds_measured = smcx.probe_lds_rate(stream) / 1e9  # G lane-loads/s
    except smcx.SmcxError:
        lds_measured = None

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local_rank)
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        lat.sweep(T_KELVIN, 1, SEED)
    e1.record(stream)
    e1.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms_max, value = aggregate_ranks(ms, WORK.sites, args.steps, dist)
    launches_per_sweep = 8 if sched[1] != (1, 1, 1) else sched[0] ** 3 * 2
    n_launch = launches_per_sweep * args.steps

    st_head = lat.state()[1]

    # ---- per-trial directions (the proposal drawn independently per trial) --
    per_trial = None
    if not args.no_site:
        lat.set_proposal(smcx.PROPOSAL_SITE)
        for _ in range(args.warmup):
            lat.sweep(T_KELVIN, 1, SEED)
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            lat.sweep(T_KELVIN, 1, SEED)
        e1.record(stream)
        e1.synchronize()
        barrier()
        ms_p, value_p = aggregate_ranks(e0.elapsed_time(e1), WORK.sites, args.steps, dist)
        lat.set_proposal(PROPOSAL)
        per_trial = {"value": value_p, "unit": UNIT, "ms_per_step": ms_p / args.steps,
                     "kernel": "k_bcc_tile_sweep<4,1,2,1,0>",
                     "frac_smem": None,
                     "note": "the same sweep with a shell-1 direction drawn per trial: same stationary "
                             "distribution, different trajectories; per-lane partner environments land on "
                             "scattered banks (about 1.84 shared-memory wavefronts per load, the shared pipe at 93% of its peak)"}

    # ---- end to end through the C ABI with host buffers -------------------
    e2e = None
    if not args.no_e2e:
        # Two handles on two streams: the upload of step i+1's input overlaps
        # the sweep of step i (double buffering); every step still uploads its
        # own input and reads back its own result (the sweep's attempt, accept
        # and summed-dE counters) inside the timed region.
        nbytes = lat.store_bytes()
        stream2 = torch.cuda.Stream()
        with torch.cuda.stream(stream2):
            lat2 = smcx.Lattice(smcx.BCC, WORK.dims, WORK.M, WORK.comp, init_seed=WORK.init_seed + rank + 7,
                                storage=smcx.PACKED4, stream=stream2)
            lat2.set_proposal(PROPOSAL)
            lat2.set_epi(V)
        hosts = [torch.empty(nbytes, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
        lat.get_config_store_ptr(hosts[0].data_ptr(), nbytes)
        lat2.get_config_store_ptr(hosts[1].data_ptr(), nbytes)
        pair = [lat, lat2]
        for i in range(2):  # warm-up of both handles
            pair[i].set_config_store_ptr(hosts[i].data_ptr(), nbytes)
            pair[i].sweep(T_KELVIN, 1, SEED)
            pair[i].state()
        barrier()
        ne = max(4, args.steps)  # the same step count as the device-timed region
        t0 = time.perf_counter()
        pair[0].set_config_store_ptr(hosts[0].data_ptr(), nbytes)   # H2D of step 0's input
        for i in range(ne):
            cur, nxt = pair[i % 2], pair[(i + 1) % 2]
            cur.sweep(T_KELVIN, 1, SEED)                              # enqueued; runs while the next upload goes
            if i + 1 < ne:
                nxt.set_config_store_ptr(hosts[(i + 1) % 2].data_ptr(), nbytes)  # H2D of step i+1's input
            cur.state()                                               # D2H of step i's result
        dt = time.perf_counter() - t0
        tt = torch.tensor([dt], device="cuda")
        if dist is not None:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dt = float(tt.item())
        e2e = {"value": WORK.sites * ne * world / dt, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": 32, "steps": ne,
               "step": "smcx_set_config_store (packed 4-bit store layout, pinned host) + smcx_sweep (1 sweep) + "
                       "smcx_get_state (attempts, accepts, same-species proposals, summed dE: 32 B); two handles "
                       "on two streams, the next step's upload overlapping this step's sweep",
               "ms_per_step": dt * 1e3 / ne}
        lat2.close()
        host = hosts
        del host

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    hbm_peak, peak_kind = peaks()
    per_launch_ms = ms_max / n_launch
    bytes_per_launch = ALG_BYTES_PER_ATTEMPT * WORK.sites / launches_per_sweep
    achieved_gbs = bytes_per_launch / (per_launch_ms / 1e3) / 1e9
    gathers_per_launch = ALG_GATHERS_PER_ATTEMPT * WORK.sites / launches_per_sweep
    lds_nominal = SM_COUNT_NOMINAL * 32 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e9  # G lane-loads/s
    lds_peak = lds_measured if lds_measured else lds_nominal
    achieved_g = gathers_per_launch / (per_launch_ms / 1e3) / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if os.path.exists(prof):
        try:
            with open(prof) as f:
                tj = json.load(f)
            # counters of the kernel timed here only
            if tj.get("kernel") == "k_bcc_tile_sweep<4,1,2,1,1>":
                traffic = tj.get("dram_bytes_per_launch")
        except Exception:
            traffic = None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": config_block({"schedule": {"L": sched[0], "tiles": list(sched[1])},
                                "parallelism": f"replicas x{world}" if world > 1 else "single lattice"}),
        "roofline": {"bound": "smem", "achieved": achieved_g, "peak": lds_peak, "unit": "Gload/s",
                     "frac": achieved_g / lds_peak, "traffic": traffic,
                     "kernel": "k_bcc_tile_sweep<4,1,2,1,1>",
                     "peak_source": "measured (smcx_probe_lds_rate: conflict-free LDS.U8 stream on every SM)"
                                    if lds_measured else "nominal (152 SMs x 32 lanes x 2070 MHz)",
                     "peak_nominal": lds_nominal,
                     "note": "shared-memory gather roof: 70 algorithmic lane-loads per trial (s, s' and the "
                             "68-site union of their environments) x trials per launch / launch time; the "
                             "kernel itself is issue-bound (see profiles/)",
                     "accept_rate": float(st_head[1]) / max(1, int(st_head[0]))},
        "roofline_hbm": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved_gbs / hbm_peak, "traffic": traffic, "peak_source": peak_kind,
                         "note": "1 B per trial (packed 4-bit read + write) per launch / launch time"},
        "gpu_launches": n_launch,
        "clocks": clk,
    }
    if e2e is not None:
        out["e2e"] = e2e
    if per_trial is not None:
        per_trial["frac_smem"] = (ALG_GATHERS_PER_ATTEMPT * WORK.sites / launches_per_sweep /
                                  (per_trial["ms_per_step"] / launches_per_sweep / 1e3) / 1e9) / lds_peak
        out["per_trial_direction"] = per_trial
    if not args.no_batched and world == 1:
        out["batched"] = run_batched(stream)
        out["replica_exchange"] = run_exchange(stream)
    if not args.no_grad and world == 1:
        out["gradient"] = run_gradient(stream)
    if not args.no_clusters and world == 1:
        out["clusters"] = run_clusters(stream)
    if not args.no_fcc and world == 1:
        out["fcc_400"] = run_fcc(stream)
    if not args.no_qsro and world == 1:
        out["qsro"] = run_qsro(stream)
    if not args.no_paper and world == 1:
        out["paper_tables"] = run_paper_rows(stream)
    if not args.no_throughput and world == 1:
        out["throughput_256"] = run_throughput256(stream)
    if not args.no_anneal and world == 1:
        out["anneal"] = run_anneal(stream)
    if not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline()
    print(json.dumps(out), flush=True)
    lat.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    global WORK
    args = parse()
    if args.dims:
        import dataclasses
        WORK = dataclasses.replace(WORK, name=f"bcc{args.dims}_q4_k4_packed4", dims=(args.dims,) * 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.impl == "reference" else 1)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if "WORLD_SIZE" not in os.environ:
        world = 1
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.only:
        import torch
        stream = torch.cuda.Stream()
        fn = {"batched": run_batched, "exchange": run_exchange, "gradient": run_gradient,
              "throughput": run_throughput256, "anneal": run_anneal, "baselines": run_baselines,
              "fcc": lambda st: run_fcc(st, args.edge), "paper": run_paper_rows,
              "clusters": lambda st: run_clusters(st, args.edge), "qsro": lambda st: run_qsro(st, args.edge),
              "batch_launch": lambda st: run_batch_launch(st, args.proposal, args.batch_sched),
              "qsro_launch": lambda st: run_qsro_launch(st, args.edge)}
        print(json.dumps({args.only: fn[args.only](stream)}), flush=True)
    else:
        run_smcx(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
