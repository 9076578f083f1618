#!/usr/bin/env python
"""Benchmark of the batched 1D-TDSE hot path on GB300.

Workload (default): the macroscopic volume batch -- 64 radial x 128 axial = 8192 independent
length-gauge TDSE instances, N = 4096 (dx = 0.15), dt = 0.02, 800 nm 10-cycle sin^2 pulse
(Nt = 55159 steps), synthetic Gaussian-beam fields, FP64, FULL_CN, cos^(1/8) mask.

One benchmark step = one tdse_propagate call that advances every instance by one chunk of
ceil(Nt / (warmup + steps)) time steps (RHS, tridiagonal solve, mask and d/a observables of every
grid point of every instance, every time step).  Warm-up plus timed steps together cover the
whole propagation exactly once, so the run also yields complete a(t) for the spectrum and the
oracle comparison.  The soft-core fit and ground state (once per grid class) and the spectrum
(once per job) are timed separately and reported beside the step throughput.

Metric: grid-point-steps/s = instances x N x time steps / seconds (whole job over all GPUs).

--impl reference runs the FP64 CPU oracle (the reference arm of this build) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2507_04115_gb300.spectral_metrics import (FP64_BOUND, MIXED_BOUND, harmonic_cutoff,  # noqa: E402
                                                    harmonic_errors_by_decades, spectral_errors)

METRIC = "1D-TDSE grid-point-steps/s (batched) & % pipe roofline; mixed vs FP64 at stated error"
UNIT = "grid-point-steps/s"
FLOPS_PER_POINT_STEP = 48.0          # algorithmic FULL_CN work per grid-point step (FMA = 2 flops)
MIXED_FP64_FLOPS_PER_POINT_STEP = 10.0   # MIXED: the FP64 pivot recurrence per grid-point step
FP64_FMA_PER_CLK_PER_SM = 2.0        # GB300 FP64 pipe: 2 FMA/clk/SM (1.2 TFLOP/s measured at 2.0 GHz)
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_propagate_full_cn_fp64_volume_traffic.txt")
KERNEL_SRCS = [os.path.join(ROOT, "paper_2507_04115_gb300", "csrc", f)
               for f in ("tdse_full_cn.cu", "tdse_sched.cuh", "tdse_device.cuh")]


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["own", "reference"], default="own")
    p.add_argument("--workload", choices=["volume", "single", "uneven", "adjoint", "large", "resolvent", "field",
                                                "populations", "hankel", "numerov"],
                   default="volume",
                   help="volume = the benchmark; the others measure the other workloads (one JSON line each)")
    p.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                   help="arithmetic of the measured path (the volume benchmark's line is fp64)")
    p.add_argument("--e2e-steps", type=int, default=2, help="chunks timed end to end through host buffers")
    p.add_argument("--cpu-baseline", type=int, default=1, help="time the oracle on the host cores (rank 0, N = 1)")
    p.add_argument("--cpu-instances", type=int, default=0, help="oracle sample size (0 = one per core, max 16)")
    p.add_argument("--ref-steps-per-step", type=int, default=4096, help="oracle time steps per reference step")
    p.add_argument("--warps", type=int, default=0, help="override warps per CTA (segments per instance)")
    p.add_argument("--ctas-per-sm", type=int, default=0, help="override CTAs per SM of the persistent grid")
    p.add_argument("--slice", type=int, default=0, help="override time steps per scheduling slice")
    p.add_argument("--autotune", type=int, default=1,
                   help="pick warps/CTAs per SM/slice with tdse_autotune before timing (untimed; 0 = planner default)")
    p.add_argument("--tune-steps", type=int, default=256, help="time steps per autotuner probe")
    p.add_argument("--instances", type=int, default=8192, help="instances per GPU (smaller = profiling case)")
    p.add_argument("--nt", type=int, default=0, help="propagate only the first nt steps (0 = whole pulse)")
    p.add_argument("--secondary", type=int, default=1,
                   help="also measure the other configurations (single atom, NUMEROV, adjoint, field ingestion) and "
                        "the analysis of the final states, as extra keys of the line")
    p.add_argument("--far-field", type=int, default=1,
                   help="also time the source spectrum and the far field (Hankel) of the volume's a(t)")
    p.add_argument("--mixed-compare", type=int, default=1,
                   help="also time the MIXED path on two chunks and propagate the oracle sample in MIXED")
    return p.parse_args()


# ------------------------------------------------------------------------------------------- helpers

def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        self.proc.wait()
        rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_sha():
    """sha256 over the sources of the FULL_CN kernel (kernel, scheduler and device helpers)."""
    h = hashlib.sha256()
    for f in KERNEL_SRCS:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def kernel_traffic_per_point_step():
    """DRAM bytes per grid-point step of k_propagate_full_cn<fp64> from the committed ncu summary, or None
    when the summary is missing or the kernel source changed since the capture."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    kv = {}
    for line in open(TRAFFIC_FILE):
        if ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    sha = kernel_source_sha()
    if kv.get("source_sha256") != sha:
        return None
    try:
        return float(kv["bytes_per_point_step"])
    except (KeyError, ValueError):
        return None


def _oracle_job(args):
    """One oracle propagation in a worker process; returns (a(t), the worker's own seconds for it)."""
    import oracle
    (psi0, E, dx, dt, a, mask, n_end) = args
    t0 = time.perf_counter()
    _, d, acc = oracle.propagate(psi0, E, dx, dt, a, mask_values=mask, n_begin=0, n_end=n_end)
    return acc, time.perf_counter() - t0


def _cpu_baseline_line(n_jobs, N, steps, secs, cores, sample):
    """Oracle throughput from the workers' own timers: every job ran in its own process on its own
    core, started together, so the sample took max(secs) of wall time on `cores` cores."""
    pts = float(N) * steps
    return {"value": n_jobs * pts / max(secs), "unit": UNIT, "cores": cores, "kind": "oracle",
            "per_core": statistics.mean(pts / s for s in secs), "sample": sample,
            "how": "sum of the sample's grid-point steps / the slowest worker's own perf_counter time around "
                   "oracle.propagate; per_core = mean over workers of their own rate"}


def run_oracle_pool(jobs, workers):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(processes=workers)
    return pool


T_AU_S = 2.4188843265857e-17      # atomic unit of time (s)
C_M_S = 299792458.0                 # speed of light (m/s)


def far_field_stage(tdse, torch, acc_rows, offs, dt, omega0, q_max, geom, stream, n_obs=256, z_obs=0.5,
                    rho_obs_max=5e-3, repeats=3):
    """The output side of the path on a volume's a(t): the source spectrum at every DFT bin with
    q <= q_max (tdse_dipole_spectrum, homogeneous density 1) and the far field of that source at
    n_obs radii of the plane z_obs (tdse_hankel).  Each call is timed with CUDA events on the
    launching stream (best of `repeats`); returns (timings dict, S, E)."""
    L = int(offs[1] - offs[0])
    k_max = int(math.floor(q_max * omega0 * L * dt / (2 * math.pi)))
    om = 2 * math.pi * np.arange(1, k_max + 1) / (L * dt)
    n_r, n_z = geom["n_r"], geom["n_z"]
    rho = np.linspace(0.0, geom["w0_m"], n_r)
    z = np.linspace(-geom["zR_m"], geom["zR_m"], n_z)
    k = om / T_AU_S / C_M_S
    ro = np.linspace(0.0, rho_obs_max, n_obs)
    n = n_r * n_z
    S = torch.empty((n, om.size), dtype=torch.complex128, device=acc_rows.device)
    E = torch.empty((om.size, n_obs), dtype=torch.complex128, device=acc_rows.device)

    def best(fn):
        ts = []
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return min(ts)

    t_s = best(lambda: tdse.dipole_spectrum(acc_rows, offs, dt, om, out=S, stream=stream))
    Sv = S.view(n_r, n_z, om.size)
    t_h = best(lambda: tdse.hankel(Sv, rho, z, k, z_obs, ro, out=E, stream=stream))
    terms = float(om.size) * n_obs * n * 1.0
    res = {"source_spectrum_ms": t_s, "hankel_ms": t_h, "frequencies": int(om.size), "q_max": q_max,
           "source_points": n, "observation_radii": n_obs, "z_obs_m": z_obs, "rho_obs_max_m": rho_obs_max,
           "hankel_terms_per_s": terms / (t_h * 1e-3),
           "source_sample_terms_per_s": float(n) * om.size * L / (t_s * 1e-3),
           "how": "CUDA events around each call, best of %d; a term = one (frequency, radius, source point) "
                  "J0-weighted product" % repeats}
    return res, S, E


# ------------------------------------------------------------------------------------------- own arm

def own_arm(args):
    import torch
    rank, world, local_rank = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)

    from paper_2507_04115_gb300 import build, inputs, softcore, tdse
    build.build()
    tdse.load()
    import oracle  # test infrastructure: used only for the CPU baseline and the spectral check
    oracle.build()

    from paper_2507_04115_gb300 import sharding
    # weak scaling: rank r owns its own 64 x 128 block of a (64 x 128 world)-point volume
    full = inputs.gaussian_beam_volume(n_z=128 * world) if world > 1 else inputs.volume_batch()
    blk = sharding.contiguous(8192 * world, world, rank)
    n = min(args.instances, blk.stop - blk.start)
    sl = slice(blk.start, blk.start + n)
    N, dx, dt = int(full.N[0]), float(full.dx[0]), full.dt
    Nt = int(full.n_steps[0]) if args.nt <= 0 else min(args.nt, int(full.n_steps[0]))
    omega, ncyc = float(full.omega[0]), float(full.n_cycles[0])
    E0, phi = full.E0[sl], full.phi[sl]
    n_chunks = args.warmup + args.steps
    S = int(math.ceil(Nt / n_chunks))
    chunks = [(c * S, min(Nt, (c + 1) * S)) for c in range(n_chunks)]

    # CPU baseline: oracle instances started now in spawned workers, running while the GPU works
    cpu_pool = cpu_async = None
    cores = 0
    sample_idx = []
    if args.cpu_baseline and rank == 0 and world == 1:
        cores = args.cpu_instances or min(16, os.cpu_count() or 1)
        sample_idx = list(inputs.subsample(n, cores, 101))

    t0 = time.time()
    a_soft = softcore.fit_softening(full.target_energy, N, dx, device=local_rank)
    t_fit = time.time() - t0

    if sample_idx:
        psi0_o, _, _ = oracle.ground_state(N, dx, a_soft)
        m = oracle.mask(N, dx, full.mask_width, full.mask_exponent)
        jobs = [(psi0_o, inputs.sin2_pulse(Nt, dt, E0[i], omega, ncyc, phi[i]), dx, dt, a_soft, m, Nt)
                for i in sample_idx]
        cpu_pool = run_oracle_pool(jobs, cores)
        cpu_async = cpu_pool.map_async(_oracle_job, jobs, chunksize=1)

    offs = np.arange(n + 1, dtype=np.int64) * (S + 1)
    main_prec = tdse.TDSE_MIXED if args.precision == "mixed" else tdse.TDSE_FP64
    batch = tdse.Batch([N] * n, dx, a_soft, [Nt] * n, dt, row_offsets=offs,
                       absorber=(full.mask_width, full.mask_exponent), precision=main_prec, device=local_rank)
    if args.warps or args.ctas_per_sm or args.slice:
        batch.set_launch(args.warps, args.ctas_per_sm, args.slice)
    plan = batch.plan()
    stream = torch.cuda.current_stream(dev)

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    batch.ground_state()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    t_gs_ms = ev0.elapsed_time(ev1)

    # device-resident chunk inputs and outputs
    Ec = []
    for (s0, s1) in chunks:
        e = torch.zeros((n, S + 1), dtype=torch.float64, device=dev)
        full_rows = torch.empty((n, s1 - s0 + 1), dtype=torch.float64, device=dev)
        tt = (torch.arange(s0, s1 + 1, dtype=torch.float64, device=dev) * dt)
        Tp = ncyc * 2 * math.pi / omega
        env = torch.where(tt <= Tp, torch.sin(math.pi * tt / Tp) ** 2, torch.zeros_like(tt))
        e0 = torch.as_tensor(E0, device=dev)
        ph = torch.as_tensor(phi, device=dev)
        full_rows.copy_(e0[:, None] * env[None, :] * torch.cos(omega * (tt[None, :] - 0.5 * Tp) + ph[:, None]))
        e[:, : s1 - s0 + 1] = full_rows
        Ec.append(e.reshape(-1))
    dc = [torch.zeros(n * (S + 1), dtype=torch.float64, device=dev) for _ in chunks]
    ac = [torch.zeros(n * (S + 1), dtype=torch.float64, device=dev) for _ in chunks]

    tune = None
    if args.autotune and not (args.warps or args.ctas_per_sm or args.slice):
        s0, s1 = chunks[0]
        trials = batch.autotune(Ec[0], dc[0], ac[0], s0, min(s1, s0 + args.tune_steps), sample_base=s0, stream=stream)
        plan = batch.plan()
        tune = dict(probe_steps=min(s1, s0 + args.tune_steps) - s0, trials=len(trials),
                    best_ms=min(t["ms"] for t in trials), default_ms=next(
                        (t["ms"] for t in trials if (t["warps_per_cta"], t["ctas_per_sm"], t["slice_steps"]) ==
                         (8 if main_prec == tdse.TDSE_FP64 else 12, 1, 16)), None))

    for c in range(args.warmup):
        s0, s1 = chunks[c]
        batch.propagate(Ec[c], dc[c], ac[c], s0, s1, sample_base=s0, stream=stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local_rank)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for k in range(args.steps):
        c = args.warmup + k
        s0, s1 = chunks[c]
        starts[k].record(stream)
        batch.propagate(Ec[c], dc[c], ac[c], s0, s1, sample_base=s0, stream=stream)
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    launch_ms = [starts[k].elapsed_time(ends[k]) for k in range(args.steps)]
    total_ms = starts[0].elapsed_time(ends[-1])
    timed_steps = sum(chunks[args.warmup + k][1] - chunks[args.warmup + k][0] for k in range(args.steps))
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    pt_steps = float(n) * N * timed_steps * world
    value = pt_steps / (total_ms * 1e-3)
    bad = batch.check(stream)

    # a(t) of the whole propagation and its spectrum (once per job)
    acc_full = torch.empty((n, Nt + 1), dtype=torch.float64, device=dev)
    for c, (s0, s1) in enumerate(chunks):
        blk = ac[c].view(n, S + 1)
        lo = 0 if c == 0 else 1
        acc_full[:, s0 + lo: s1 + 1] = blk[:, lo: s1 - s0 + 1]
    q_cut = harmonic_cutoff(float(np.max(E0)), omega)
    L = Nt + 1
    k_max = min(L, int(math.ceil(1.5 * q_cut * omega * L * dt / (2 * math.pi))) + 2)
    ev0.record(stream)
    S_dev = tdse.spectrum(acc_full.reshape(-1), np.arange(n + 1) * L, dt, 0, k_max, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    t_spec_ms = ev0.elapsed_time(ev1)

    # analysis of the final states (Sec. 6.1, 7.5): energy distribution, ionisation probability and
    # populations of every instance after the whole pulse, on the benchmark batch itself
    analysis = None
    if world == 1 and args.secondary:
        clk_a = ClockSampler(local_rank)
        clk_a.start()
        E_grid = np.linspace(-0.7, 2.5, 128)
        P = torch.empty((n, E_grid.size), dtype=torch.float64, device=dev)
        t_ed = _timed(torch, dev, stream, lambda: batch.energy_distribution(E_grid, 0.02, out=P, stream=stream))
        nodes = np.linspace(0.0, 2.5, 401)
        ion = torch.empty(n, dtype=torch.float64, device=dev)
        t_ion = _timed(torch, dev, stream, lambda: batch.ionisation(nodes, 0.02, out=ion, stream=stream))
        pops = torch.empty((n, 2), dtype=torch.float64, device=dev)
        batch.populations(2.0, out=pops, stream=stream)
        t_pop = _timed(torch, dev, stream, lambda: batch.populations(2.0, out=pops, stream=stream))
        ion_h, pop_h = ion.cpu().numpy(), pops.cpu().numpy()
        analysis = {"energy_distribution": {"solves_per_s": n * E_grid.size / t_ed, "seconds": t_ed,
                                            "energies": int(E_grid.size), "eps": 0.02},
                    "ionisation": {"solves_per_s": n * nodes.size / t_ion, "seconds": t_ion, "nodes": int(nodes.size),
                                   "range_au": [0.0, 2.5], "eps": 0.02, "min": float(ion_h.min()),
                                   "max": float(ion_h.max())},
                    "populations": {"states_per_s": n / t_pop, "seconds": t_pop, "r_core": 2.0,
                                    "ground_population_range": [float(pop_h[:, 0].min()), float(pop_h[:, 0].max())]},
                    "state": "every instance after the whole %d-step pulse" % Nt, "clocks": clk_a.stop()}

    # the output side on this volume's a(t): source spectrum and far field (Sec. 3.2, 4.3)
    far = None
    if world == 1 and args.far_field:
        far, _, _ = far_field_stage(tdse, torch, acc_full.reshape(-1), np.arange(n + 1) * L, dt, omega,
                                    1.5 * q_cut, full.extra, stream)

    # end to end: host (pinned) field chunks in, d and a chunks out, through the public binding
    e2e = None
    if args.e2e_steps > 0:
        batch.ground_state()
        n_e2e = min(args.e2e_steps, n_chunks)
        Eh = [Ec[c].cpu().pin_memory() for c in range(n_e2e)]
        dh = [torch.empty(n * (S + 1), dtype=torch.float64).pin_memory() for _ in range(n_e2e)]
        ah = [torch.empty(n * (S + 1), dtype=torch.float64).pin_memory() for _ in range(n_e2e)]
        # one untimed pass warms torch's caching allocator for the binding's device copies
        batch.propagate(Eh[0], dh[0], ah[0], chunks[0][0], chunks[0][1], sample_base=chunks[0][0], stream=stream)
        batch.ground_state()
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        e0_ = torch.cuda.Event(enable_timing=True)
        e1_ = torch.cuda.Event(enable_timing=True)
        e0_.record(stream)
        for c in range(n_e2e):
            s0, s1 = chunks[c]
            batch.propagate(Eh[c], dh[c], ah[c], s0, s1, sample_base=s0, stream=stream)
        e1_.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = e0_.elapsed_time(e1_)
        if world > 1:
            t = torch.tensor([e2e_ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_ms = float(t.item())
        e2e_pts = float(n) * N * sum(chunks[c][1] - chunks[c][0] for c in range(n_e2e)) * world
        e2e = {"value": e2e_pts / (e2e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(n * (S + 1) * 8), "d2h_bytes_per_step": int(2 * n * (S + 1) * 8),
               "steps": n_e2e, "how": "Batch.propagate with pinned CPU tensors: H2D field chunk, kernel, "
                                     "D2H d and a chunks, CUDA events on the launching stream"}

    # CPU baseline results and spectral error of the sampled instances
    cpu_baseline = None
    spec_err = None
    if cpu_async is not None:
        res = cpu_async.get()
        cpu_pool.close()
        cpu_pool.join()
        accs = [r[0] for r in res]
        secs = [r[1] for r in res]
        cpu_baseline = _cpu_baseline_line(len(sample_idx), N, Nt, secs, cores,
                                          "%d instances of this workload (seeded subsample), full %d-step propagation "
                                          "each, one spawned process per core" % (len(sample_idx), Nt))
        S_host = S_dev.cpu().numpy()
        acc_host = acc_full.cpu().numpy()
        l2s, worst, byd = [], [], {}
        series = 0.0
        for j, i in enumerate(sample_idx):
            S_ref = oracle.spectrum(accs[j], dt)[:k_max]
            l2, w = spectral_errors(S_host[i], S_ref, omega, dt, L, q_cut)
            l2s.append(l2)
            worst.append(w)
            for D, e in harmonic_errors_by_decades(S_host[i], S_ref, omega, dt, L, q_cut).items():
                byd[D] = max(byd.get(D, 0.0), e)
            series = max(series, float(np.max(np.abs(acc_host[i] - accs[j])) / np.max(np.abs(accs[j]))))
        spec_err = {"instances": len(sample_idx), "rel_l2_max": max(l2s), "harmonic_rel_max": max(worst),
                    "harmonic_rel_max_within_decades": byd, "a_series_rel_max": series, "q_cut": q_cut,
                    "bound": list(FP64_BOUND)}

    # mixed precision on the same workload: throughput over two chunks of the whole batch, and the
    # spectral error of the oracle sample propagated in full (one group, so it runs on one SM)
    mixed = None
    if args.mixed_compare and world == 1 and main_prec == tdse.TDSE_FP64:
        batch.close()
        mb = tdse.Batch([N] * n, dx, a_soft, [Nt] * n, dt, row_offsets=offs,
                        absorber=(full.mask_width, full.mask_exponent), precision=tdse.TDSE_MIXED, device=local_rank)
        mb.ground_state()
        m_tune = None
        if args.autotune:
            s0, s1 = chunks[0]
            mt = mb.autotune(Ec[0], dc[0], ac[0], s0, min(s1, s0 + args.tune_steps), sample_base=s0, stream=stream)
            mp = mb.plan()
            m_tune = dict(warps_per_cta=mp["warps_per_cta"], ctas=mp["ctas"], slice_steps=mp["slice_steps"],
                          trials=len(mt))
        n_m = max(1, min(2, n_chunks - 1))   # chunks after the first (untimed) one
        mb.propagate(Ec[0], dc[0], ac[0], chunks[0][0], chunks[0][1], sample_base=chunks[0][0], stream=stream)
        torch.cuda.synchronize(dev)
        e0_ = torch.cuda.Event(enable_timing=True)
        e1_ = torch.cuda.Event(enable_timing=True)
        e0_.record(stream)
        timed_m = [c for c in range(1, 1 + n_m) if c < n_chunks] or [0]
        for c in timed_m:
            s0, s1 = chunks[c]
            mb.propagate(Ec[c], dc[c], ac[c], s0, s1, sample_base=s0, stream=stream)
        e1_.record(stream)
        torch.cuda.synchronize(dev)
        m_ms = e0_.elapsed_time(e1_)
        m_val = float(n) * N * sum(chunks[c][1] - chunks[c][0] for c in timed_m) / (m_ms * 1e-3)
        mixed = {"value": m_val, "unit": UNIT, "speedup_vs_fp64": m_val / value, "steps": n_m, "launch": m_tune,
                 "dtype": "psi f32, elimination recurrence and observable sums f64"}
        mb.close()
        if cpu_async is not None:
            k = len(sample_idx)
            Es = torch.from_numpy(np.concatenate([inputs.sin2_pulse(Nt, dt, E0[i], omega, ncyc, phi[i])
                                                  for i in sample_idx])).to(dev)
            ms_ = tdse.Batch([N] * k, dx, a_soft, [Nt] * k, dt, absorber=(full.mask_width, full.mask_exponent),
                             precision=tdse.TDSE_MIXED, device=local_rank)
            ms_.ground_state()
            dm, am = torch.zeros_like(Es), torch.zeros_like(Es)
            ms_.propagate(Es, dm, am, stream=stream)
            Sm = tdse.spectrum(am, np.arange(k + 1) * L, dt, 0, k_max, stream=stream).cpu().numpy()
            ms_.close()
            l2s, worst, byd = [], [], {}
            for j in range(k):
                S_ref = oracle.spectrum(accs[j], dt)[:k_max]
                l2, wv = spectral_errors(Sm[j], S_ref, omega, dt, L, q_cut)
                l2s.append(l2)
                worst.append(wv)
                for D, e in harmonic_errors_by_decades(Sm[j], S_ref, omega, dt, L, q_cut).items():
                    byd[D] = max(byd.get(D, 0.0), e)
            mixed["spectral_error"] = {"instances": k, "rel_l2_max": max(l2s), "harmonic_rel_max": max(worst),
                                       "harmonic_rel_max_within_decades": byd, "bound": list(MIXED_BOUND)}

    # the other configurations and rows, bounded so that the whole line stays within a few minutes
    secondary = None
    if world == 1 and args.secondary:
        secondary = {}
        for name, fn in (("single_atom", lambda: measure_single(torch, tdse, inputs, softcore, dev, stream, 1, 1, 2)),
                         ("numerov_volume", lambda: measure_numerov(torch, tdse, inputs, softcore, dev, stream, 300, 1)),
                         ("adjoint_batch", lambda: measure_adjoint(torch, tdse, inputs, softcore, dev, stream, 0, 1, 128,
                                                                   plain=False)),
                         ("field_ingestion", lambda: measure_field(torch, tdse, inputs, dev, stream))):
            ck = ClockSampler(local_rank)
            ck.start()
            r = fn()
            r["clocks"] = ck.stop()
            secondary[name] = r
        secondary["analysis_of_final_states"] = analysis

    avg_launch_s = statistics.mean(launch_ms) * 1e-3
    pts_per_launch = float(n) * N * (timed_steps / args.steps)
    # FP64 work per point-step: the whole step in FP64; in MIXED only the pivot recurrence of the
    # elimination stays on the FP64 pipe (10 flops + the reciprocal)
    fp64_flops = FLOPS_PER_POINT_STEP if main_prec == tdse.TDSE_FP64 else MIXED_FP64_FLOPS_PER_POINT_STEP
    achieved = fp64_flops * pts_per_launch / avg_launch_s
    peak = FP64_FMA_PER_CLK_PER_SM * 2 * SM_COUNT * SM_MAX_MHZ * 1e6
    tpp = kernel_traffic_per_point_step() if main_prec == tdse.TDSE_FP64 else None
    pipes = tdse.tdse_probe_pipes(local_rank)
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": (tpp * pts_per_launch) if tpp is not None else None,
                "kernel": "k_propagate_full_cn<%s>" % args.precision, "pipe": "fp64",
                "peak_how": "2 FP64 FMA/clk/SM x 152 SMs x 2 flops x 2070 MHz (unit counts at max clock)",
                "fp64_fma_measured_tflops": pipes["fp64_fma_tflops"],
                "achieved_how": "%g FP64 flops per grid-point step x points x steps per launch / mean CUDA-event "
                                "launch time" % fp64_flops}
    if mixed is not None:
        # the MIXED kernel against the FP32 pipe (the algorithmic 48 flops), with the share that stays
        # on the FP64 pipe (the pivot recurrence) against the FP64 peak
        m_ach = FLOPS_PER_POINT_STEP * mixed["value"]
        m_fp64 = MIXED_FP64_FLOPS_PER_POINT_STEP * mixed["value"]
        mixed["roofline"] = {
            "bound": "alu", "pipe": "fp32 (fp64 share stated)", "achieved": m_ach / 1e12,
            "peak": pipes["fp32_fma_tflops"], "unit": "TFLOP/s", "frac": m_ach / 1e12 / pipes["fp32_fma_tflops"],
            "traffic": None, "kernel": "k_propagate_full_cn<mixed>",
            "peak_how": "FP32 FMA rate measured by tdse_probe_pipes on this GPU",
            "fp64_share": {"flops_per_point_step": MIXED_FP64_FLOPS_PER_POINT_STEP, "achieved": m_fp64 / 1e12,
                           "peak": peak / 1e12, "frac": m_fp64 / peak},
            "achieved_how": "%g flops per grid-point step x grid-point-steps/s over the timed MIXED chunks "
                            "(CUDA events)" % FLOPS_PER_POINT_STEP}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if main_prec == tdse.TDSE_FP64 else "f32 psi / f64 elimination and sums",
           "data": "synthetic",
           "config": {"workload": "volume batch 64r x 128z = 8192 instances per GPU, N=4096 dx=0.15, dt=0.02, "
                                  "800 nm 10-cycle sin^2 Gaussian-beam fields, FP64 FULL_CN, cos^(1/8) mask",
                      "instances_per_gpu": n, "N": N, "dx": dx, "dt": dt, "Nt": Nt, "chunk_steps": S,
                      "step": "one tdse_propagate call advancing every instance by chunk_steps time steps",
                      "l2": "inputs larger than L2: psi %.0f MB + scratch %.0f MB per GPU" %
                            (plan["psi_bytes"] / 1e6, plan["scratch_bytes"] / 1e6),
                      "precision": args.precision, "scheme": "full_cn", "segments": plan["segments"],
                      "halo": plan["halo"], "warps_per_cta": plan["warps_per_cta"], "ctas": plan["ctas"],
                      "slice_steps": plan["slice_steps"], "autotune": tune,
                      "parallelism": "instances sharded over GPUs, no collective"},
           "solves_per_s": value / (N * Nt),
           "roofline": roofline, "cpu_baseline": cpu_baseline, "e2e": e2e, "clocks": clk,
           "gpu_launches": args.steps, "nonfinite_instance": bad,
           "setup": {"softening_fit_s": t_fit, "softening": a_soft, "ground_state_ms": t_gs_ms,
                     "spectrum_ms": t_spec_ms, "spectrum_bins": k_max},
           "spectral_error": spec_err, "mixed": mixed, "far_field": far, "secondary": secondary}
    if rank == 0:
        print(json.dumps(out), flush=True)
    batch.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------------------------------- reference arm

def reference_arm(args):
    """The FP64 CPU oracle on the host cores: each step propagates a bounded sample of the same
    workload (one instance per core, ref-steps-per-step time steps each)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp
    import oracle
    from paper_2507_04115_gb300 import inputs
    oracle.build()
    wl = inputs.volume_batch()
    N, dx, dt = int(wl.N[0]), float(wl.dx[0]), wl.dt
    Nt = int(wl.n_steps[0])
    cores = args.cpu_instances or min(16, os.cpu_count() or 1)
    T = min(Nt, args.ref_steps_per_step)
    a = oracle.fit_softening(wl.target_energy, N, dx)
    psi0, _, _ = oracle.ground_state(N, dx, a)
    m = oracle.mask(N, dx, wl.mask_width, wl.mask_exponent)
    idx = inputs.subsample(wl.n_inst, cores, 101)
    jobs = [(psi0, inputs.sin2_pulse(T, dt, wl.E0[i], float(wl.omega[0]), float(wl.n_cycles[0]), wl.phi[i]), dx, dt,
             a, m, T) for i in idx]
    ctx = mp.get_context("spawn")
    times = []
    with ctx.Pool(processes=cores) as pool:
        for k in range(args.warmup + args.steps):
            t0 = time.time()
            pool.map(_oracle_job, jobs, chunksize=1)
            if k >= args.warmup:
                times.append(time.time() - t0)
    pts = float(len(jobs)) * N * T
    total = sum(times)
    value = pts * len(times) / total
    sample = ("%d instances x %d steps of the volume batch per step (seeded subsample), one spawned process per "
              "core" % (len(jobs), T))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / len(times) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "volume batch 64r x 128z = 8192 instances, N=4096 dx=0.15, dt=0.02, 800 nm "
                                  "10-cycle sin^2 Gaussian-beam fields, FP64 FULL_CN, cos^(1/8) mask",
                      "N": N, "dx": dx, "dt": dt, "Nt": Nt, "sample": sample},
           "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": value, "unit": UNIT},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------------------------------- other workloads

def _measured_hbm_gbs():
    """Measured HBM copy bandwidth of this GPU type in GB/s (MEASURED_PEAKS.json beside this file),
    else the 6.8 TB/s fallback measured earlier on a GB300."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def _line(metric, value, unit, args, workload, cfg, **extra):
    out = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
           "config": dict(workload=workload, **cfg)}
    out.update(extra)
    print(json.dumps(out), flush=True)


def _fit(softcore, wl_target, classes, dev_index):
    return {c: softcore.fit_softening(wl_target, c[0], c[1], device=dev_index) for c in classes}


def other_workload(args):
    """Single atom, uneven batch, adjoint batch and large volume: measured for the record, one line each."""
    import torch
    from paper_2507_04115_gb300 import build, inputs, softcore, tdse
    build.build()
    tdse.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    prec = tdse.TDSE_MIXED if args.precision == "mixed" else tdse.TDSE_FP64

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) * 1e-3

    if args.workload == "single":
        r = measure_single(torch, tdse, inputs, softcore, dev, stream, args.autotune, args.warmup, args.steps)
        _line(METRIC, r["fp64"], UNIT, args, r["workload"], r["config"], dtype="f64",
              mixed={"value": r["mixed"], "speedup_vs_fp64": r["mixed"] / r["fp64"]},
              solves_per_s=r["fp64"] / r["points_per_solve"],
              note="the instance spans the lanes of one CTA's warps (lane-split layout, one SM)")
        return

    if args.workload == "numerov":
        r = measure_numerov(torch, tdse, inputs, softcore, dev, stream, args.nt or 300, args.autotune)
        _line(METRIC, r["fp64"]["value"], UNIT, args, r["workload"], r["config"], dtype="f64", mixed=r["mixed"],
              fp64=r["fp64"])
        return

    if args.workload == "uneven":
        uneven_full(args, torch, tdse, inputs, softcore, dev)
        return

    if args.workload == "large":
        large_stream(args, torch, tdse, inputs, softcore, dev)
        return

    if args.workload == "field":
        # field ingestion (Sec. 4.2): 8192 coarse rows of 2400 samples at 0.5 a.u. (a 1200 a.u. window
        # around the 10-cycle pulse) interpolated to the volume batch's 55160 samples at dt = 0.02
        wl = inputs.volume_batch()
        n = wl.n_inst if args.instances <= 0 else min(args.instances, wl.n_inst)
        M, dt_c, dt_f = 2400, 0.5, wl.dt
        n_fine = int(wl.n_steps[0]) + 1
        coarse = torch.empty((n, M - 1), dtype=torch.float64, device=dev)
        inputs.sin2_pulse_batch(M - 2, dt_c, wl.E0[:n], float(wl.omega[0]), float(wl.n_cycles[0]), wl.phi[:n],
                                out=coarse, xp=torch)
        coarse = torch.cat([coarse, torch.zeros((n, 1), dtype=torch.float64, device=dev)], dim=1).contiguous()
        out = torch.empty((n, n_fine), dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            tdse.resample_field(coarse, dt_c, dt_f, n_fine, out=out)
        ts = [timed(lambda: tdse.resample_field(coarse, dt_c, dt_f, n_fine, out=out)) for _ in range(args.steps)]
        t = statistics.mean(ts)
        _line("field ingestion samples/s (Sec. 4.2, zero-padded DFT interpolation)", float(n) * n_fine / t,
              "fine samples/s", args, "%d rows x %d coarse samples (dt %g) -> %d samples (dt %g)" % (n, M, dt_c, n_fine, dt_f),
              dict(rows=n, M=M, dt_coarse=dt_c, dt_fine=dt_f, n_fine=n_fine), dtype="f64",
              fp64_instructions_per_sample=6 * (M // 2 + 1), seconds_per_call=t)
        return

    if args.workload == "populations":
        # ground-state population and near-core probability (Sec. 7.5) of the volume batch's states
        # after a chunk of the pulse.  The kernel reads the rows in the hull of the ground state's
        # support (tails below 1e-17) and of |x| < r_core; the same rule is applied here to the
        # ground state to count the bytes it has to read.  Those rows (tens of MB) fit in L2, so
        # a 512 MB buffer is read before every timed call (a read leaves no dirty lines to write back).
        wl = inputs.volume_batch()
        n = wl.n_inst if args.instances <= 0 else min(args.instances, wl.n_inst)
        N, dx, dt = int(wl.N[0]), float(wl.dx[0]), wl.dt
        a = softcore.fit_softening(wl.target_energy, N, dx)
        Nt = 200 if args.nt <= 0 else args.nt
        E = torch.empty((n, Nt + 1), dtype=torch.float64, device=dev)
        inputs.sin2_pulse_batch(Nt, dt, wl.E0[:n], float(wl.omega[0]), float(wl.n_cycles[0]), wl.phi[:n], out=E, xp=torch)
        E = E.reshape(-1).contiguous()
        b = tdse.Batch([N] * n, dx, a, [Nt] * n, dt, absorber=(wl.mask_width, wl.mask_exponent), precision=prec)
        b.ground_state()
        r_core = 2.0
        w0 = np.abs(b.get_psi(0).cpu().numpy()) ** 2 * dx
        thr = 0.5e-34
        s_lo = int(np.searchsorted(np.cumsum(w0), thr, side="right"))
        s_hi = N - int(np.searchsorted(np.cumsum(w0[::-1]), thr, side="right"))
        x = (np.arange(N) - 0.5 * (N - 1)) * dx
        core = np.nonzero(np.abs(x) < r_core)[0]
        rows = max(s_hi, int(core[-1]) + 1) - min(s_lo, int(core[0]))
        d, acc = torch.zeros_like(E), torch.zeros_like(E)
        b.propagate(E, d, acc)
        out = torch.empty((n, 2), dtype=torch.float64, device=dev)
        flush = torch.ones(64 << 20, dtype=torch.float64, device=dev)
        sink = torch.empty((), dtype=torch.float64, device=dev)
        for _ in range(max(args.warmup, 3)):
            b.populations(r_core, out=out)
        ev = []
        torch.cuda.synchronize(dev)
        for _ in range(args.steps):
            torch.sum(flush, dim=0, out=sink)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.populations(r_core, out=out)
            e1.record(stream)
            ev.append((e0, e1))
        torch.cuda.synchronize(dev)
        t = statistics.mean(e0.elapsed_time(e1) * 1e-3 for e0, e1 in ev)
        b.close()
        cx = 16 if prec == tdse.TDSE_FP64 else 8
        bytes_ = float(n) * rows * cx + 16.0 * n
        # the FP64 pipe bounds it: two FP64 FMAs per point read (the overlap's real and imaginary
        # parts), two more per core point; the rows themselves need less time from HBM
        flops = 4.0 * n * rows + 4.0 * n * int(core.size)
        peak = FP64_FMA_PER_CLK_PER_SM * 2 * SM_COUNT * SM_MAX_MHZ * 1e6
        _line("state populations per second (Sec. 7.5)", n / t, "instance states/s", args,
              "populations of the volume batch: %d instances, N=%d, r_core=%g, after %d steps" % (n, N, r_core, Nt),
              dict(instances=n, N=N, r_core=r_core, steps_before=Nt, precision=args.precision, rows_read=rows,
                   core_rows=int(core.size), l2="512 MB read before every timed call"),
              dtype="f64 sums", seconds_per_call=t, gpu_launches=args.steps,
              hbm={"achieved": bytes_ / t / 1e9, "peak": _measured_hbm_gbs(), "unit": "GB/s",
                   "frac": bytes_ / t / 1e9 / _measured_hbm_gbs(),
                   "how": "rows_read rows of every state (%d B per point) plus the 16 B result per instance" % cx},
              roofline={"bound": "alu", "achieved": flops / t / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                        "frac": flops / t / peak, "traffic": None,
                        "achieved_how": "2 FP64 FMAs per point of the rows read, 2 more per core point"})
        return

    if args.workload == "resolvent":
        # energy distribution (Sec. 6.1) of the volume batch's states after a chunk of the pulse:
        # 8192 instances x 128 energies, each a complex tridiagonal solve over N = 4096 points
        wl = inputs.volume_batch()
        n = wl.n_inst if args.instances <= 0 else min(args.instances, wl.n_inst)
        N, dx, dt = int(wl.N[0]), float(wl.dx[0]), wl.dt
        a = softcore.fit_softening(wl.target_energy, N, dx)
        Nt = 2000 if args.nt <= 0 else args.nt
        E = torch.empty((n, Nt + 1), dtype=torch.float64, device=dev)
        inputs.sin2_pulse_batch(Nt, dt, wl.E0[:n], float(wl.omega[0]), float(wl.n_cycles[0]), wl.phi[:n], out=E, xp=torch)
        E = E.reshape(-1).contiguous()
        b = tdse.Batch([N] * n, dx, a, [Nt] * n, dt, absorber=(wl.mask_width, wl.mask_exponent), precision=prec)
        b.ground_state()
        d, acc = torch.zeros_like(E), torch.zeros_like(E)
        b.propagate(E, d, acc)
        n_E, eps = 128, 0.02
        E_grid = np.linspace(-0.7, 2.5, n_E)
        P = torch.empty((n, n_E), dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            b.energy_distribution(E_grid, eps, out=P)
        ts = [timed(lambda: b.energy_distribution(E_grid, eps, out=P)) for _ in range(args.steps)]
        t = statistics.mean(ts)
        solves = float(n) * n_E
        flops = 22.0 * solves * N   # per point: r - a d' 4, times 1/w 6, y = d' - c'y 8, |y|^2 4
        b.close()
        peak = FP64_FMA_PER_CLK_PER_SM * 2 * SM_COUNT * SM_MAX_MHZ * 1e6
        _line("energy-distribution resolvent solves/s (Sec. 6.1)", solves / t, "tridiagonal solves/s", args,
              "energy distribution of the volume batch: %d instances x %d energies, N=%d, eps=%g, after %d steps"
              % (n, n_E, N, eps, Nt),
              dict(instances=n, energies=n_E, N=N, eps=eps, steps_before=Nt, precision=args.precision),
              dtype="f64", point_solves_per_s=solves * N / t,
              roofline={"bound": "alu", "achieved": flops / t / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                        "frac": flops / t / peak, "traffic": None,
                        "achieved_how": "22 FP64 flops per point of each (instance, energy) solve; the pivot "
                                        "pass per (class, energy) is amortised and not counted"})
        return

    if args.workload == "hankel":
        # the output side at the volume batch's shape: 8192 dipole-acceleration rows of 55160
        # samples (synthetic: odd harmonics of 800 nm with seeded amplitudes and phases under the
        # pulse's sin^2 envelope), their source spectrum at every bin up to 1.5 q_cut, and the far
        # field of the 64 x 128 source points at 256 radii
        wl = inputs.volume_batch()
        n, dt, Nt = wl.n_inst, wl.dt, int(wl.n_steps[0])
        omega = float(wl.omega[0])
        L = Nt + 1
        rng = np.random.default_rng(7)
        t = torch.arange(L, dtype=torch.float64, device=dev) * dt
        Tp = float(wl.n_cycles[0]) * 2 * math.pi / omega
        env = torch.sin(math.pi * t / Tp) ** 2
        acc = torch.zeros((n, L), dtype=torch.float64, device=dev)
        for q in range(1, 40, 2):
            amp = torch.from_numpy(rng.uniform(0.5, 1.5, n) * 10.0 ** (-0.1 * q)).to(dev)
            ph = torch.from_numpy(rng.uniform(0, 2 * math.pi, n)).to(dev)
            acc += amp[:, None] * env[None, :] * torch.cos(q * omega * t[None, :] + ph[:, None])
        q_cut = harmonic_cutoff(float(np.max(wl.E0)), omega)
        res, _, _ = far_field_stage(tdse, torch, acc.reshape(-1), np.arange(n + 1) * L, dt, omega, 1.5 * q_cut,
                                    wl.extra, stream, repeats=max(1, args.steps))
        _line("far-field (Hankel) terms/s (Sec. 3.2 Eq. Hankel long homogeneous, Sec. 4.3)",
              res["hankel_terms_per_s"], "terms/s", args,
              "far field of the volume batch's source: 64 r x 128 z points, %d frequencies, %d radii"
              % (res["frequencies"], res["observation_radii"]),
              dict(res, rows=n, samples_per_row=L,
                   a_rows="synthetic: seeded odd harmonics under the sin^2 envelope, the volume batch's shape"),
              dtype="f64", gpu_launches=2 * max(1, args.steps))
        return

    if args.workload == "adjoint":
        r = measure_adjoint(torch, tdse, inputs, softcore, dev, stream, args.nt, args.autotune, args.tune_steps,
                            n_inst=args.instances if args.instances < 1024 else 0)
        cfg = r.pop("config")
        _line("1D-TDSE adjoint gradient, forward-equivalent grid-point-steps/s", r.pop("value"), UNIT, args,
              r.pop("workload"), cfg, dtype="f64", **r)
        return


def _timed(torch, dev, stream, fn):
    """Seconds of fn's GPU work: CUDA events on the launching stream, synchronised on both sides."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) * 1e-3


def measure_single(torch, tdse, inputs, softcore, dev, stream, autotune=1, warmup=1, steps=3):
    """The single atom (N = 2000, 8818 steps): whole propagations in FP64 and MIXED (best layout)."""
    wl = inputs.single_atom()
    N, dx, dt = int(wl.N[0]), float(wl.dx[0]), wl.dt
    a = softcore.fit_softening(wl.target_energy, N, dx)
    E = torch.from_numpy(wl.field_rows()[0]).to(dev)
    Nt = E.numel() - 1
    res, shapes = {}, {}
    for pname, pv in (("fp64", tdse.TDSE_FP64), ("mixed", tdse.TDSE_MIXED)):
        b = tdse.Batch([N], dx, a, [Nt], dt, absorber=(wl.mask_width, wl.mask_exponent), precision=pv)
        d, acc = torch.zeros_like(E), torch.zeros_like(E)
        b.ground_state()
        if autotune:
            b.autotune(E, d, acc, 0, min(Nt, 512))
        shapes[pname] = dict((k, b.plan()[k]) for k in ("lanes_per_instance", "warps_per_cta", "segments", "halo"))
        ts = []
        for k in range(warmup + steps):
            b.ground_state()
            t = _timed(torch, dev, stream, lambda: b.propagate(E, d, acc))
            if k >= warmup:
                ts.append(t)
        res[pname] = float(N) * Nt / statistics.mean(ts)
        b.close()
    return {"fp64": res["fp64"], "mixed": res["mixed"], "points_per_solve": N * Nt,
            "workload": "single atom N=2000 dx=0.2 dt=0.05, 800 nm 4-cycle sin^2, 8818 steps",
            "config": dict(N=N, dx=dx, dt=dt, Nt=Nt, step="one whole propagation of the single instance", layout=shapes)}


def measure_numerov(torch, tdse, inputs, softcore, dev, stream, steps=300, autotune=1):
    """The paper's scheme (NUMEROV_SPLIT, Sec. 4.2) on the volume batch's shape: 8192 x 4096 over the
    first `steps` steps, FP64 and MIXED, the soft-core a fitted on the Numerov H0."""
    wl = inputs.volume_batch()
    n, N, dx, dt = wl.n_inst, int(wl.N[0]), float(wl.dx[0]), wl.dt
    a = softcore.fit_softening(wl.target_energy, N, dx, scheme=tdse.TDSE_NUMEROV_SPLIT)
    E = torch.empty((n, steps + 1), dtype=torch.float64, device=dev)
    inputs.sin2_pulse_batch(steps, dt, wl.E0, float(wl.omega[0]), float(wl.n_cycles[0]), wl.phi, out=E, xp=torch)
    E = E.reshape(-1).contiguous()
    out = {}
    for pname, pv in (("fp64", tdse.TDSE_FP64), ("mixed", tdse.TDSE_MIXED)):
        b = tdse.Batch([N] * n, dx, a, [steps] * n, dt, absorber=(wl.mask_width, wl.mask_exponent), precision=pv,
                       scheme=tdse.TDSE_NUMEROV_SPLIT)
        b.ground_state()
        d, acc = torch.zeros_like(E), torch.zeros_like(E)
        if autotune:
            b.autotune(E, d, acc, 0, min(steps, 64))
        b.ground_state()
        t = _timed(torch, dev, stream, lambda: b.propagate(E, d, acc))
        plan = b.plan()
        out[pname] = {"value": float(n) * N * steps / t, "seconds": t, "nonfinite_instance": b.check(),
                      "launch": dict((k, plan[k]) for k in ("warps_per_cta", "ctas", "slice_steps", "segments", "halo"))}
        b.close()
    out["mixed"]["speedup_vs_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    out["workload"] = "NUMEROV_SPLIT (Sec. 4.2) on the volume batch: 8192 x 4096, first %d steps" % steps
    out["config"] = dict(instances=n, N=N, dx=dx, dt=dt, steps=steps, scheme="numerov_split")
    return out


def measure_adjoint(torch, tdse, inputs, softcore, dev, stream, nt=0, autotune=1, tune_steps=256, plain=True,
                    n_inst=0):
    """The adjoint batch (1024 x 2048, 6 cycles): the forward propagation, the checkpointed forward
    (recording a checkpoint every 256 steps) and the adjoint gradient of the harmonic 21-31 yield
    from those checkpoints, each timed once; with `plain`, also tdse_adjoint, which runs its own
    forward pass.  n_inst > 0 takes the first n_inst instances only, laid out as in the whole
    batch (4 lanes per instance): a profiling case with fewer groups and tapes."""
    wl = inputs.adjoint_batch()
    n = wl.n_inst if n_inst <= 0 else min(n_inst, wl.n_inst)
    N, dx, dt = int(wl.N[0]), float(wl.dx[0]), wl.dt
    Nt = int(wl.n_steps[0]) if nt <= 0 else nt
    a = softcore.fit_softening(wl.target_energy, N, dx)
    E = torch.empty((n, Nt + 1), dtype=torch.float64, device=dev)
    inputs.sin2_pulse_batch(Nt, dt, wl.E0[:n], float(wl.omega[0]), float(wl.n_cycles[0]), wl.phi[:n], out=E, xp=torch)
    E = E.reshape(-1).contiguous()
    b = tdse.Batch([N] * n, dx, a, [Nt] * n, dt, absorber=(wl.mask_width, wl.mask_exponent),
                   lanes_per_instance=4 if n < wl.n_inst else 0)
    b.ground_state()
    d, acc = torch.zeros_like(E), torch.zeros_like(E)
    if autotune:
        b.autotune(E, d, acc, 0, min(Nt, tune_steps))
    psi0 = b.save_state()
    t_fwd = _timed(torch, dev, stream, lambda: b.propagate(E, d, acc))
    b.load_state(psi0)
    # loss = harmonic yield of q in [21, 31]: dL/da from the spectrum of every row
    L = Nt + 1
    q = np.fft.fftfreq(L, dt) * 2 * np.pi / float(wl.omega[0])
    win = torch.from_numpy(((np.abs(q) >= 21) & (np.abs(q) <= 31)).astype(np.float64)).to(dev)
    A = torch.fft.fft(acc.view(n, L), dim=1)
    ga = (2 * dt * dt * torch.fft.ifft(A * win[None, :], dim=1).real * L).reshape(-1).contiguous()
    gd = torch.zeros_like(E)
    t_rec = _timed(torch, dev, stream, lambda: b.propagate_checkpointed(E, d, acc, 256))
    t_adj = _timed(torch, dev, stream, lambda: b.adjoint_checkpointed(E, gd, ga))
    out = {}
    if plain:
        b.load_state(psi0)
        t_plain = _timed(torch, dev, stream, lambda: b.adjoint(E, gd, ga, ckpt_every=256))
        out = {"self_contained_adjoint_s": t_plain, "self_contained_over_forward_time": t_plain / t_fwd}
    pts = float(n) * N * Nt
    layout = dict((k, b.plan()[k]) for k in ("lanes_per_instance", "warps_per_cta", "segments", "halo", "ctas"))
    b.close()
    out.update({"value": pts / t_adj, "forward_value": pts / t_fwd, "adjoint_over_forward_time": t_adj / t_fwd,
                "recording_over_forward_time": t_rec / t_fwd, "gradient_total_over_forward_time": (t_rec + t_adj) / t_fwd,
                "forward_s": t_fwd, "recording_forward_s": t_rec, "adjoint_s": t_adj, "workload": wl.name,
                "how": "adjoint_s: tdse_adjoint_checkpointed after tdse_propagate_checkpointed (the autograd "
                       "backward); value = forward-equivalent point-steps per second of that backward pass",
                "config": dict(instances=n, N=N, Nt=Nt, ckpt_every=256,
                               loss="sum of dt^2|DFT(a)|^2 over harmonics 21-31", layout=layout)})
    return out


def measure_field(torch, tdse, inputs, dev, stream, rows=2048, repeats=2):
    """Field ingestion (Sec. 4.2) of the volume batch's rows: 2400 coarse samples at 0.5 a.u. ->
    55160 samples at dt = 0.02 (best of `repeats`)."""
    wl = inputs.volume_batch()
    n = min(rows, wl.n_inst)
    M, dt_c, dt_f = 2400, 0.5, wl.dt
    n_fine = int(wl.n_steps[0]) + 1
    coarse = torch.empty((n, M - 1), dtype=torch.float64, device=dev)
    inputs.sin2_pulse_batch(M - 2, dt_c, wl.E0[:n], float(wl.omega[0]), float(wl.n_cycles[0]), wl.phi[:n],
                            out=coarse, xp=torch)
    coarse = torch.cat([coarse, torch.zeros((n, 1), dtype=torch.float64, device=dev)], dim=1).contiguous()
    out = torch.empty((n, n_fine), dtype=torch.float64, device=dev)
    tdse.resample_field(coarse, dt_c, dt_f, n_fine, out=out)
    t = min(_timed(torch, dev, stream, lambda: tdse.resample_field(coarse, dt_c, dt_f, n_fine, out=out))
            for _ in range(repeats))
    return {"value": float(n) * n_fine / t, "unit": "fine samples/s", "seconds_per_call": t, "rows": n, "M": M,
            "n_fine": n_fine, "fp64_instructions_per_sample": 6 * (M // 2 + 1)}


# ------------------------------------------------------------------------------------------- configuration-size runs

def _oracle_pool(wl, idx, soft_of_inst):
    """The oracle's whole-pulse propagation of instances idx, started now in spawned processes (one per
    core); returns (pool, async result, cores).  The ground state and mask are computed once per class."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    cache, jobs = {}, []
    for i in idx:
        N, dx = int(wl.N[i]), float(wl.dx[i])
        if (N, dx) not in cache:
            psi0, _, _ = oracle.ground_state(N, dx, float(soft_of_inst[i]))
            cache[(N, dx)] = (psi0, oracle.mask(N, dx, wl.mask_width, wl.mask_exponent))
        psi0, m = cache[(N, dx)]
        jobs.append((psi0, wl.field_rows([i])[0], dx, wl.dt, float(soft_of_inst[i]), m, int(wl.n_steps[i])))
    cores = max(1, min(len(jobs), os.cpu_count() or 1))
    pool = mp.get_context("spawn").Pool(processes=cores)
    return pool, pool.map_async(_oracle_job, jobs, chunksize=1), cores


def _pulse_params(torch, wl, dev):
    """Per-instance pulse parameters as device columns (E0, omega, Tp, phi), made before any capture."""
    return tuple(torch.as_tensor(v, dtype=torch.float64, device=dev)[:, None]
                 for v in (wl.E0, wl.omega, wl.n_cycles * 2 * np.pi / wl.omega, wl.phi))


def _fill_rows(torch, E, prm, dt, s0, S, dev):
    """Field samples n = s0 .. s0 + S of every instance into E (rows of S + 1 samples), on the device:
    E0 sin^2(pi t/Tp) cos(w (t - Tp/2) + phi) for t <= Tp, 0 after; prm from _pulse_params.  Device
    work only, so it can be captured in a CUDA graph."""
    e0, w, Tp, ph = prm
    t = (torch.arange(s0, s0 + S + 1, dtype=torch.float64, device=dev) * dt)[None, :]
    env = torch.where(t <= Tp, torch.sin(np.pi * t / Tp) ** 2, torch.zeros_like(t))
    E.view(e0.shape[0], S + 1).copy_(e0 * env * torch.cos(w * (t - 0.5 * Tp) + ph))


def _fill_full_rows(torch, E, offs, wl, dev, block=256):
    """Whole-pulse rows of every instance (row i: Nt_i + 1 samples at offs[i]), by blocks of instances."""
    n = wl.n_inst
    for b0 in range(0, n, block):
        b1 = min(n, b0 + block)
        lens = torch.as_tensor(offs[b0 + 1: b1 + 1] - offs[b0: b1], device=dev)
        idx = torch.repeat_interleave(torch.arange(b0, b1, device=dev), lens)
        start = torch.repeat_interleave(torch.as_tensor(offs[b0: b1], device=dev), lens)
        t = (torch.arange(int(offs[b0]), int(offs[b1]), device=dev) - start).to(torch.float64) * wl.dt
        prm = [torch.as_tensor(v, device=dev)[idx] for v in (wl.E0, wl.omega, wl.n_cycles * 2 * np.pi / wl.omega, wl.phi)]
        e0, w, Tp, ph = prm
        env = torch.where(t <= Tp, torch.sin(np.pi * t / Tp) ** 2, torch.zeros_like(t))
        E[int(offs[b0]): int(offs[b1])] = e0 * env * torch.cos(w * (t - 0.5 * Tp) + ph)


def _sample_errors(tdse, wl, idx, rows_gpu, refs, dev):
    """Spectral errors (relative L2 over q <= 1.5 q_cut, worst odd harmonic) of the sampled instances'
    a(t) rows against the oracle's; the GPU spectra come from tdse_spectrum."""
    import oracle
    import torch
    l2s, hs, byd = [], [], {}
    for j, i in enumerate(idx):
        a_row = rows_gpu[j]
        L = a_row.numel()
        S = tdse.spectrum(a_row.to(dev).contiguous(), [0, L], wl.dt, 0, L).cpu().numpy()[0]
        S_ref = oracle.spectrum(refs[j], wl.dt)
        omega = float(wl.omega[i])
        qc = harmonic_cutoff(float(wl.E0[i]), omega)
        l2, h = spectral_errors(S, S_ref, omega, wl.dt, L, qc)
        l2s.append(l2)
        hs.append(h)
        for D, e in harmonic_errors_by_decades(S, S_ref, omega, wl.dt, L, qc).items():
            byd[D] = max(byd.get(D, 0.0), e)
    return {"instances": len(idx), "rel_l2_max": max(l2s), "harmonic_rel_max": max(hs),
            "harmonic_rel_max_within_decades": byd}


def uneven_full(args, torch, tdse, inputs, softcore, dev):
    """The uneven batch (16384 instances, N 1024..8192, up to 198575 steps) through the whole pulse
    of every instance, FP64 then MIXED: fields resident on the device, one persistent launch over
    every step of every instance (or one per chunk of --nt steps), captured once in a CUDA graph and
    replayed (timed); spectral error of the oracle sample (64 instances, seed 102) on the run's own
    a(t).  One launch lets the scheduler run the longest groups from the start (a launch per chunk
    waits at every chunk's end for its longest group)."""
    wl = inputs.uneven_batch()
    n = wl.n_inst
    classes = sorted(set(zip(wl.N.tolist(), wl.dx.tolist())))
    soft = _fit(softcore, wl.target_energy, classes, 0)
    a = np.array([soft[(int(N_), float(d_))] for N_, d_ in zip(wl.N, wl.dx)])
    nt = wl.n_steps.astype(np.int64)
    offs = np.concatenate([[0], np.cumsum(nt + 1)]).astype(np.int64)
    Nt_max = int(nt.max())
    sample = inputs.subsample(n, 64, 102) if args.cpu_baseline else np.array([], dtype=np.int64)
    pool = res = None
    cores = 0
    if sample.size:
        pool, res, cores = _oracle_pool(wl, sample, a)
    E = torch.empty(int(offs[-1]), dtype=torch.float64, device=dev)
    _fill_full_rows(torch, E, offs, wl, dev)
    S = int(args.nt) if args.nt > 0 else Nt_max   # default: the whole job in one persistent launch
    chunks = [(s0, min(Nt_max, s0 + S)) for s0 in range(0, Nt_max, S)]
    pts = wl.point_steps()
    out, rows = {}, {}
    for pname, prec in (("fp64", tdse.TDSE_FP64), ("mixed", tdse.TDSE_MIXED)):
        b = tdse.Batch(wl.N, wl.dx, a, nt, wl.dt, row_offsets=offs, absorber=(wl.mask_width, wl.mask_exponent),
                       precision=prec)
        b.ground_state()
        d, acc = torch.zeros_like(E), torch.zeros_like(E)
        if args.autotune:
            b.autotune(E, d, acc, 0, args.tune_steps, sample_base=0)
        b.propagate(E, d, acc, 0, 1)           # the launch path once outside the capture
        b.ground_state()
        torch.cuda.synchronize(dev)
        st = torch.cuda.Stream(dev)
        st.wait_stream(torch.cuda.current_stream(dev))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            for (s0, s1) in chunks:
                b.propagate(E, d, acc, s0, s1, sample_base=0, stream=st)
        clocks = ClockSampler(0)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):            # replay() launches on the current stream
            e0.record(st)
            g.replay()
            e1.record(st)
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        sec = e0.elapsed_time(e1) * 1e-3
        plan = b.plan()
        out[pname] = {"value": pts / sec, "seconds": sec, "clocks": clk, "nonfinite_instance": b.check(),
                      "launch": dict((k, plan[k]) for k in ("warps_per_cta", "ctas", "slice_steps", "segments", "halo"))}
        rows[pname] = [acc[int(offs[i]): int(offs[i + 1])].clone() for i in sample]
        b.close()
        del g
    if pool is not None:
        got = res.get()
        refs = [r[0] for r in got]
        pool.close()
        pool.join()
        for pname in out:
            out[pname]["spectral_error"] = _sample_errors(tdse, wl, sample, rows[pname], refs, dev)
        oracle_pts = float(np.sum(wl.N[sample].astype(np.float64) * nt[sample]))
        out["cpu_baseline"] = {"value": oracle_pts / max(r[1] for r in got), "unit": UNIT, "cores": cores,
                               "kind": "oracle", "sample": "the 64-instance oracle sample, whole pulses"}
    _line(METRIC, out["fp64"]["value"], UNIT, args, wl.name,
          dict(instances=n, classes=len(classes), Nt_max=Nt_max, chunk_steps=S, chunks=len(chunks),
               steps_covered="every step of every instance", precision="fp64 (mixed in 'mixed')",
               graph="the launch sequence captured once in a CUDA graph and replayed",
               l2="fields, d and a resident: %.1f GB each" % (offs[-1] * 8 / 1e9)),
          dtype="f64", total_point_steps=pts, solves_per_s=n / out["fp64"]["seconds"],
          fp64=out["fp64"], mixed=dict(out["mixed"], speedup_vs_fp64=out["mixed"]["value"] / out["fp64"]["value"]),
          gpu_launches=len(chunks), bound={"fp64": list(FP64_BOUND), "mixed": list(MIXED_BOUND)},
          cpu_baseline=out.get("cpu_baseline"))


def large_stream(args, torch, tdse, inputs, softcore, dev):
    """The large volume (131072 x 4096, MIXED, 1800 nm, 99288 steps) streamed by chunks of steps: the
    field chunk synthesised on the device, the propagation, and the a(t) chunk copied to pinned host
    memory on a second stream (double-buffered, overlapping the next chunk), the timed chunks captured
    once in a CUDA graph and replayed.  The 32 instances of the oracle sample (seed 104) also run
    the whole pulse in a batch of their own with the same launch layout: their a(t) over the timed
    chunks must equal the large batch's bit for bit, and their spectra are compared with the oracle."""
    wl = inputs.large_volume()
    n, N, dt = wl.n_inst, int(wl.N[0]), wl.dt
    Nt = int(wl.n_steps[0])
    a_soft = softcore.fit_softening(wl.target_energy, N, float(wl.dx[0]))
    S = int(args.nt) if args.nt > 0 else 2000
    n_warm, n_timed = max(1, args.warmup), max(1, args.steps)
    sample = inputs.subsample(n, 32, 104)
    pool = res = None
    if args.cpu_baseline:
        pool, res, _ = _oracle_pool(wl, sample, np.full(n, a_soft))
    offs = np.arange(n + 1, dtype=np.int64) * (S + 1)
    b = tdse.Batch(wl.N, wl.dx, a_soft, wl.n_steps, dt, row_offsets=offs, absorber=(wl.mask_width, wl.mask_exponent),
                   precision=tdse.TDSE_MIXED)
    b.ground_state()
    Ec = [torch.zeros(int(offs[-1]), dtype=torch.float64, device=dev) for _ in range(2)]
    dc = [torch.zeros_like(Ec[0]) for _ in range(2)]
    ac = [torch.zeros_like(Ec[0]) for _ in range(2)]
    hb = [torch.empty(int(offs[-1]), dtype=torch.float64).pin_memory() for _ in range(2)]
    sample_dev = torch.as_tensor(sample, device=dev)
    prm = _pulse_params(torch, wl, dev)
    gathered = torch.zeros((n_timed, sample.size, S + 1), dtype=torch.float64, device=dev)
    if args.autotune:
        _fill_rows(torch, Ec[0], prm, dt, 0, S, dev)
        b.autotune(Ec[0], dc[0], ac[0], 0, min(S, args.tune_steps), sample_base=0)
        b.ground_state()
    plan = b.plan()
    main = torch.cuda.current_stream(dev)
    for c in range(n_warm):                     # eager warm-up chunks (the first steps of the pulse)
        _fill_rows(torch, Ec[c % 2], prm, dt, c * S, S, dev)
        b.propagate(Ec[c % 2], dc[c % 2], ac[c % 2], c * S, (c + 1) * S, sample_base=c * S)
        hb[c % 2].copy_(ac[c % 2], non_blocking=True)
    torch.cuda.synchronize(dev)
    st, cs = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    st.wait_stream(main)
    # one captured graph per timed chunk (field synthesis on the device and the persistent launch),
    # sharing one memory pool; the copy-back is not captured: it runs on the copy stream between
    # the replays, double-buffered (chunk c + 2 reuses chunk c's buffers once its copy is done)
    graphs = []
    gpool = None
    for k in range(n_timed):
        c = n_warm + k
        s0 = c * S
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st, pool=gpool):
            _fill_rows(torch, Ec[c % 2], prm, dt, s0, S, dev)
            b.propagate(Ec[c % 2], dc[c % 2], ac[c % 2], s0, s0 + S, sample_base=s0, stream=st)
        gpool = g.pool()
        graphs.append(g)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    copy_done = {}
    with torch.cuda.stream(st):
        e0.record(st)
        for k, g in enumerate(graphs):
            c = n_warm + k
            if c - 2 in copy_done:
                st.wait_event(copy_done[c - 2])
            g.replay()
            done = torch.cuda.Event()
            done.record(st)
            cs.wait_event(done)
            with torch.cuda.stream(cs):
                hb[c % 2].copy_(ac[c % 2], non_blocking=True)
                gathered[k].copy_(ac[c % 2].view(n, S + 1).index_select(0, sample_dev))
                ev = torch.cuda.Event()
                ev.record(cs)
            copy_done[c] = ev
        st.wait_stream(cs)
        e1.record(st)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    sec = e0.elapsed_time(e1) * 1e-3
    bad = b.check()
    b.close()
    timed_pts = float(n) * N * n_timed * S
    # the oracle sample through the whole pulse with the large batch's layout (32-wide groups, same
    # warps and slice): the same arithmetic per instance as inside the large batch
    k_s = sample.size
    # the same device synthesis as the chunks (bit-identical samples): whole rows of Nt + 1 samples
    so = np.arange(k_s + 1, dtype=np.int64) * (Nt + 1)
    Es = torch.empty(int(so[-1]), dtype=torch.float64, device=dev)
    sd = torch.as_tensor(sample, device=dev)
    _fill_rows(torch, Es, tuple(p.index_select(0, sd) for p in prm), dt, 0, Nt, dev)
    bs = tdse.Batch(wl.N[sample], wl.dx[sample], a_soft, wl.n_steps[sample], dt, row_offsets=so,
                    absorber=(wl.mask_width, wl.mask_exponent), precision=tdse.TDSE_MIXED, lanes_per_instance=1)
    bs.set_launch(plan["warps_per_cta"], 1, plan["slice_steps"])
    bs.ground_state()
    ds, as_ = torch.zeros_like(Es), torch.zeros_like(Es)
    bs.propagate(Es, ds, as_)
    torch.cuda.synchronize(dev)
    bs.close()
    a_rows = [as_[int(so[j]): int(so[j + 1])] for j in range(k_s)]
    same = all(torch.equal(gathered[k, j, 1:], a_rows[j][(n_warm + k) * S + 1: (n_warm + k + 1) * S + 1])
               for k in range(n_timed) for j in range(k_s))
    spec = None
    if pool is not None:
        refs = [r[0] for r in res.get()]
        pool.close()
        pool.join()
        spec = _sample_errors(tdse, wl, sample, a_rows, refs, dev)
    _line(METRIC, timed_pts / sec, UNIT, args, wl.name,
          dict(instances=n, N=N, Nt=Nt, chunk_steps=S, warmup_chunks=n_warm, timed_chunks=n_timed,
               timed_fraction_of_pulse=n_timed * S / Nt, precision="mixed",
               pipeline="per chunk: a captured CUDA graph (field synthesised on the device, tdse_propagate) "
                        "replayed on the compute stream, then the a(t) chunk copied to double-buffered pinned "
                        "host memory on a second stream while the next chunk's graph runs",
               launch=dict((k, plan[k]) for k in ("warps_per_cta", "ctas", "slice_steps", "segments", "halo"))),
          dtype="f32 psi / f64 elimination and sums", clocks=clk, nonfinite_instance=bad,
          total_point_steps=wl.point_steps(), d2h_bytes_per_chunk=int(offs[-1]) * 8,
          sample_matches_large_batch_bitwise=bool(same), spectral_error=spec, bound=list(MIXED_BOUND),
          gpu_launches=n_timed)


def main():
    args = parse_args()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload != "volume":
        other_workload(args)
    else:
        own_arm(args)


if __name__ == "__main__":
    main()
