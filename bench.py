#!/usr/bin/env python3
"""Benchmark of the decorated-particle (Scovel-Weinstein, k = 2) step on GB300.

Prints ONE JSON line.  Default workload: bump-on-tail at bandwidth-roofline
scale, 4096 x 4096 lattice = 16,777,216 decorated particles, nx 1024, dt 0.05,
FP32 particle state, FP64 Poisson normalisation and compensated energy sums
(diagnostics every step).  A step is one pass of the whole hot path: element
keys, the stable sort (at the autotuned cadence), the fused push + deposit,
the per-run neutralisation + solve + table rebuild, and the diagnostics.

  python bench.py [--steps K] [--warmup W] [--impl ours|reference] [--gpus N]

--impl reference times the FP64 CPU oracle on the host cores (each step one
oracle step on a bounded sample of the same workload).  Under torchrun
(N > 1) every rank advances its own independent replica (weak scaling, no
collective on the data path); the time is the maximum over ranks.
"""
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "decorated particle-steps/s & % HBM roofline; batched vs plain at equal error"
UNIT = "decorated particle-steps/s"
# algorithmic bytes per particle-step of the fused pass: read Q,P,q*,p*,psi*, write Q,P,q*,p*
BYTES_PER_PARTICLE = {(32, True): 36, (64, True): 72, (32, False): 20, (64, False): 40}
FALLBACK_HBM_GBS = 6800.0
# FP64 arithmetic of one decorated particle-step of the fused pass (FMA = 2):
# element of Q (3), two half-kicks (5 each), diagnostic densities and their
# compensated sums (13), drift (4), element, coordinate and node weights of
# the deposit (10), the two shared-memory adds (2); without decoration the q*,
# p* terms drop out
FP64_FLOPS_PER_PARTICLE = {True: 42, False: 28}
FP64_NOMINAL_TFLOPS = 1.25
D2_MODES = {"lumped": 0, "nodal": 2, "p2": 3}      # swpic_d2_mode values


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--deposit-mode", choices=["atomic", "deterministic"], default="atomic")
    ap.add_argument("--diag-every", type=int, default=1)
    ap.add_argument("--resort", type=int, default=-1, help="-1: autotune")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the deterministic-mode, e2e, ensemble and CPU-baseline legs")
    ap.add_argument("--side", type=int, default=None,
                    help="lattice side (default: the workload's own, 4096 for bump_on_tail)")
    ap.add_argument("--launch", default=None, help="TPBxBPSM: fixed launch shape (no autotune)")
    ap.add_argument("--stages", type=int, default=None, help="bulk-copy stages (0 = register loads; no autotune)")
    ap.add_argument("--only-2d", action="store_true",
                    help="run only the 2D2V leg (K timed steps) and print its JSON object")
    ap.add_argument("--only-sort", action="store_true",
                    help="run only the sort leg (the main line's workload) and print its JSON object")
    ap.add_argument("--side-2d", type=int, default=4096,
                    help="2D leg: particles = side^2 = (lattice side)^4 (4096 = the 2D workload, 64^4)")
    ap.add_argument("--workload", choices=["bump_on_tail", "landau_strong", "landau_strong_pic"],
                    default="bump_on_tail",
                    help="the main line's workload (bump_on_tail = the 4096^2 benchmark workload; "
                         "landau_strong = the 2048^2 strong-Landau lattice; landau_strong_pic = its "
                         "8192^2 point-particle form)")
    ap.add_argument("--precision", type=int, choices=[32, 64], default=32,
                    help="particle-state precision of the main line")
    ap.add_argument("--d2-mode", choices=list(D2_MODES), default="lumped",
                    help="phi'' of the kick: P1 field with a lumped or nodal projection, or the P2 field")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def job_time_ms(ms, world, device):
    """The job's time over replicas: the slowest rank's (an all-reduce MAX of
    one float on `device`; no collective when world == 1)."""
    if world <= 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(world, particles_per_rank, steps, ms):
    """Whole-job throughput: every rank advances its own replica of
    particles_per_rank particles for `steps` steps within the job time."""
    return world * particles_per_rank * steps / (ms / 1e3)


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (no MEASURED_PEAKS.json)"


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f,
                stderr=subprocess.DEVNULL)
            time.sleep(0.15)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), float(parts[2]), parts[3:]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        smax = max(r[1] for r in rows)
        pmax = max(r[2] for r in rows)
        loaded = [r for r in rows if r[2] > 0.5 * pmax] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": smax,
                "power_w_max": pmax, "samples": len(rows), "samples_under_load": len(loaded),
                "reasons": reasons}


def gpu_index_for_smi(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            return vis.split(",")[dev]
        return dev


# --------------------------------------------------------------------------
# oracle legs (host cores)
# --------------------------------------------------------------------------
def oracle_sample_spec(spec, cols):
    """The workload with `cols` lattice columns instead of all: same domain,
    velocity lattice, mesh and dt, fewer particles (a bounded CPU sample)."""
    import dataclasses
    return dataclasses.replace(spec.lattice, nq=cols)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def time_oracle(spec, cols, steps, warmup, diag_every, d2_mode=0, threads=1):
    """Seconds for `steps` oracle steps on a `cols`-column sample.  Each oracle
    run factorises its dense Poisson matrix once at set-up; a step is timed as
    [t(M + 1 steps) - t(1 step)] / M, which leaves that one-time cost out.
    For the P1 fields M = max(steps, 50) and each time is the best of two
    runs, so that the steps outweigh the run-to-run spread of the
    factorisation; the P2 field solves a dense system every step (seconds a
    step, far above that spread): M = steps, one run each.  Returns
    (particles, seconds for `steps` steps, threads used, M)."""
    import oracle as O
    used = O.set_threads(threads)
    m, reps = (steps, 1) if d2_mode == 3 else (max(steps, 50), 2)
    try:
        lat = oracle_sample_spec(spec, cols)
        st = O.init_lattice(lat)
        if warmup > 0:
            st = O.run(st, spec.nx, lat.L, spec.dt, warmup, diag_every=diag_every, d2_mode=d2_mode,
                       decorated=spec.decorated)

        def run_s(k):
            best = 1e30
            for _ in range(reps):
                t0 = time.perf_counter()
                O.run(st, spec.nx, lat.L, spec.dt, k, diag_every=diag_every, d2_mode=d2_mode,
                      decorated=spec.decorated)
                best = min(best, time.perf_counter() - t0)
            return best

        t_one = run_s(1)
        t_many = run_s(m + 1)
    finally:
        O.set_threads(1)
    per_step = (t_many - t_one) / m
    if per_step <= 0.0:                     # spread larger than the steps: bound from above
        per_step = t_many / (m + 1)
    return lat.n, per_step * steps, used, m


def run_reference(args, spec):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    cols = max(1, min(spec.lattice.nq, 256))          # 256 x 4096 = 1,048,576 particles per step
    d2 = D2_MODES[args.d2_mode]
    # the oracle's P2 field is a dense (2 nx + 1)^2 solve every step: a few steps only
    steps = min(args.steps, 5) if d2 == 3 else args.steps
    warm = min(args.warmup, 1) if d2 == 3 else args.warmup
    n, dt, cores, m = time_oracle(spec, cols, steps, warm, args.diag_every, d2, threads=host_cores())
    value = n * steps / dt
    sample = ("%d of %d lattice columns (%d particles) of %s, after %d warm-up steps, plain-C FP64 "
              "oracle, particle loops on %d host threads; seconds per step = [t(M+1 steps) - "
              "t(1 step)]/M with M = %d%s (the one-time dense LU of each oracle run left out)" %
              (cols, spec.lattice.nq, n, spec.name, warm, cores, m,
               "" if d2 == 3 else ", each the best of two runs"))
    config = dict(workload_config(spec, args, None),
                  sample={"lattice_columns": cols, "particles": n, "steps": steps,
                          "note": "each step of the oracle arm is one oracle step of this sample of "
                                  "the workload; value = sample particles x steps / time"})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(spec, args, resort):
    es = 4 if spec.precision == 32 else 8
    n_arr = 5 if spec.decorated else 3
    return {"workload": spec.name, "particles": spec.lattice.n, "lattice": [spec.lattice.nq, spec.lattice.nv],
            "nx": spec.nx, "dt": spec.dt, "L": spec.lattice.L,
            "precision": "fp%d state, fp64 solve" % spec.precision, "decorated": spec.decorated,
            "deposit_mode": args.deposit_mode, "d2_mode": args.d2_mode, "diag_every": args.diag_every,
            "resort_every": resort,
            "l2": "inputs larger than L2 (state %.0f MB > 129 MB)" % (spec.lattice.n * es * n_arr / 1e6),
            "parallelism": "replicas (one independent run per GPU)"}


# --------------------------------------------------------------------------
def main():
    args = parse()
    if args.workload == "bump_on_tail":
        spec = W.bump_on_tail(precision=args.precision, side=args.side or 4096)
    else:
        import dataclasses
        spec = W.landau_strong(precision=args.precision, scale=4 if args.workload.endswith("pic") else 1,
                               decorated=not args.workload.endswith("pic"))
        if args.side:
            lat_ = dataclasses.replace(spec.lattice, nq=args.side, nv=args.side)
            spec = dataclasses.replace(spec, lattice=lat_, name="landau_strong_%dx%d%s" % (
                args.side, args.side, "" if spec.decorated else "_pic"))
    if args.impl == "reference":
        run_reference(args, spec)
        return
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if args.only_2d:
        from paper_2605_21794_gb300 import build, swpic
        build.build()
        if rank == 0:
            print(json.dumps(two_d_leg(torch, swpic, args)), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2605_21794_gb300 import build, swpic
    build.build()
    lat = spec.lattice
    n = lat.n
    prec, dec = spec.precision, spec.decorated
    mode = 1 if args.deposit_mode == "deterministic" else 0
    jx, jv = W.jitter(lat) if lat.jitter else (None, None)

    def make(mode_, resort, graphs=True):
        s = swpic.Simulation([(lat.L, spec.dt, spec.nx, n)], precision=prec, decorated=dec,
                             deposit_mode=mode_, d2_mode=D2_MODES[args.d2_mode],
                             resort_every=max(resort, 0), use_graphs=graphs, diag_capacity=64)
        s.init_lattice(0, lat, jx, jv)
        swpic.swpic_refresh(s.ctx)
        return s

    sim = make(mode, args.resort)
    # every leg starts from the initial state: the decorations of this workload
    # grow without bound late in the run, so no leg runs past
    # warm-up + K steps from t = 0
    torch.cuda.synchronize()
    arrays = lambda s: [t for t in (s.Q, s.P, s.qs, s.ps, s.psi) if t is not None]
    init_state = [t.clone() for t in arrays(sim)]

    def restore(s):
        torch.cuda.synchronize()
        for dst, src in zip(arrays(s), init_state):
            dst.copy_(src)
        torch.cuda.synchronize()
        swpic.swpic_refresh(s.ctx)

    if args.launch:
        tpb_, bpsm_ = (int(x) for x in args.launch.lower().split("x"))
        swpic.swpic_set_launch(sim.ctx, tpb_, bpsm_, max(args.resort, 0))
    if args.stages is not None:
        swpic.swpic_set_pipeline(sim.ctx, args.stages)
    fixed = args.launch is not None or args.stages is not None
    if args.resort < 0 and not args.no_autotune and not fixed:
        # tune on the state the timed region starts from (after the W warm-up
        # steps), over trials as long as the timed region (at most 50 steps);
        # the autotuner restores that state, and the run restarts from t = 0
        sim.step(args.warmup, args.diag_every)
        swpic.swpic_autotune(sim.ctx, max(5, min(args.steps, 50)), None)
    tpb, bpsm, resort = swpic.swpic_get_launch(sim.ctx)
    stages = swpic.swpic_get_pipeline(sim.ctx)[1]
    restore(sim)
    if args.only_sort:
        if rank == 0:
            print(json.dumps(sort_leg(torch, swpic, sim, n, args, (tpb, bpsm, resort), restore, arrays)),
                  flush=True)
        sim.close()
        return

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(s, k):
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(k, args.diag_every)
        e1.record(s.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        barrier()
        return ms

    # warm-up (also captures the step graphs)
    sim.step(args.warmup, args.diag_every)
    swpic.swpic_synchronize(sim.ctx)
    l0 = swpic.swpic_launch_count(sim.ctx)
    sampler = ClockSampler(gpu_index_for_smi(torch, local)) if rank == 0 else None
    if sampler:
        sampler.start()
    ms = timed(sim, args.steps)
    clocks = sampler.stop() if sampler else None
    launches = swpic.swpic_launch_count(sim.ctx) - l0
    swpic.swpic_synchronize(sim.ctx)
    ms = job_time_ms(ms, world, "cuda")
    value = job_value(world, n, args.steps, ms)

    # per-pass device durations (CUDA events on the context stream, plain launches),
    # over the same warm-up + K steps from the initial state
    restore(sim)
    sim.step(args.warmup, args.diag_every)
    swpic.swpic_set_timing(sim.ctx, 1)
    sim.step(args.steps, args.diag_every)
    pass_ms = swpic.swpic_pass_times(sim.ctx)
    swpic.swpic_set_timing(sim.ctx, 0)
    full = pass_ms[1:-1] if len(pass_ms) > 2 else pass_ms
    avg_pass_ms = float(np.mean(full))
    bpp = BYTES_PER_PARTICLE[(prec, dec)]
    achieved = bpp * n / (avg_pass_ms / 1e3) / 1e9
    peak, peak_src = measured_peak()
    main_line = args.workload == "bump_on_tail" and prec == 32 and (args.side or 4096) == 4096
    traffic = (profiled_traffic("k_pass_p2_bump_on_tail_4096" if args.d2_mode == "p2" else
                                "k_pass_bump_on_tail_4096") if main_line else None)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "k_pass<%s, %s, %s, deposit, diag%s>" % (
                    "float" if prec == 32 else "double", "decorated" if dec else "point",
                    args.deposit_mode, ", P2" if args.d2_mode == "p2" else ""),
                "algorithmic_bytes_per_launch": bpp * n,
                "avg_launch_ms": avg_pass_ms, "peak_source": peak_src,
                "step_frac": (bpp * n * world / (ms / args.steps / 1e3) / 1e9) / peak}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f%d" % prec, "data": "synthetic",
            "config": dict(workload_config(spec, args, resort),
                           launch={"threads_per_block": tpb, "blocks_per_sm": bpsm,
                                   "bulk_copy_stages": stages}),
            "roofline": roofline, "gpu_launches": int(launches), "clocks": clocks}

    if not args.no_extras and rank == 0 and main_line:
        # deterministic deposit mode, same workload
        other = 1 - mode
        s2 = make(other, resort)
        swpic.swpic_set_launch(s2.ctx, tpb, bpsm, resort)
        swpic.swpic_set_pipeline(s2.ctx, stages)
        s2.step(args.warmup, args.diag_every)
        ms2 = timed(s2, args.steps)
        line["other_deposit_mode"] = {
            "deposit_mode": "deterministic" if other == 1 else "atomic",
            "value": n * args.steps / (ms2 / 1e3), "ms_per_step": ms2 / args.steps}
        s2.close()
        restore(sim)
        line["e2e"] = e2e_leg(torch, swpic, sim, n, args)
        line["batched_vs_plain"] = ensemble_leg(torch, swpic)
        line["init_kmeans"] = kmeans_leg(torch, swpic)
        if args.d2_mode != "p2":
            line["p2_elements"] = p2_leg(torch, swpic, spec, args, (tpb, bpsm, resort, stages), timed)
        line["two_d"] = two_d_leg(torch, swpic, args)
        line["strong_landau"] = method_legs(torch, swpic, args, timed)
        line["fp32_diag_error"] = fp32_diag_error_leg(torch, swpic, spec, args)
        line["sort"] = sort_leg(torch, swpic, sim, n, args, (tpb, bpsm, resort), restore, arrays)
        line["cpu_baseline"] = cpu_baseline_leg(spec, args)
    elif rank == 0:
        restore(sim)
        line["e2e"] = e2e_leg(torch, swpic, sim, n, args)
    sim.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def profiled_traffic(name="k_pass_bump_on_tail_4096"):
    """DRAM bytes per launch of the fused pass from the committed ncu summary,
    valid only while the kernel source is the one that was profiled."""
    import hashlib
    summ = os.path.join(ROOT, "profiles", name + ".json")
    try:
        with open(summ) as f:
            d = json.load(f)
        src = os.path.join(ROOT, "paper_2605_21794_gb300", "csrc", d.get("source", "pass.cu"))
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if d.get("pass_cu_sha256") == h:
            return d.get("dram_bytes_per_launch_full_size")
    except Exception:
        pass
    return None


def e2e_leg(torch, swpic, sim, n, args):
    """The same K steps through swpic_step_host: pinned host state in, final
    state out, copies inside the timed region.  The input is the state after
    the W warm-up steps, so the K steps are the same segment of the run that
    the device-timed value covers (sim is at the initial state on entry)."""
    sim.step(args.warmup, args.diag_every)
    st = sim.state()
    npdt, tdt = (np.float32, torch.float32) if sim.precision == 32 else (np.float64, torch.float64)
    ins = ("Q", "P", "qs", "ps", "psi") if sim.decorated else ("Q", "P", "psi")
    outs = ("Q", "P", "qs", "ps") if sim.decorated else ("Q", "P")
    hin = {k: torch.from_numpy(st[k].astype(npdt)).pin_memory() for k in ins}
    hout = {k: torch.empty(n, dtype=tdt).pin_memory() for k in outs}
    p = lambda d, k: d[k].data_ptr() if k in d else None

    def call(k_steps):
        swpic.swpic_step_host(sim.ctx, p(hin, "Q"), p(hin, "P"), p(hin, "qs"), p(hin, "ps"), p(hin, "psi"),
                              p(hout, "Q"), p(hout, "P"), p(hout, "qs"), p(hout, "ps"), n, k_steps,
                              args.diag_every)
    call(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    call(args.steps)
    dt = time.perf_counter() - t0
    es = 4 if sim.precision == 32 else 8
    return {"value": n * args.steps / dt, "unit": UNIT,
            "h2d_bytes_per_step": es * len(ins) * n / args.steps,
            "d2h_bytes_per_step": es * len(outs) * n / args.steps,
            "note": "swpic_step_host on the state after the W warm-up steps: H2D of the %d state "
                    "arrays, field set-up, K steps, D2H of %d arrays, all inside the timed region" %
                    (len(ins), len(outs))}


def sort_leg(torch, swpic, sim, n, args, launch, restore, arrays):
    """The stable sort by element (Sec. 5's deposit wants particles grouped by
    element; histogram -> scan -> stable scatter into the sort buffer), timed
    as the step runs it: a re-sort before every full pass, plain launches
    with CUDA events around each pass on the context stream.  The device time
    of the whole call (events on the same stream) minus the passes' own times
    is the span of the sort kernels between them, per sort.  One sort moves
    44 B per FP32 decorated particle: the histogram reads Q, the scatter reads
    the five arrays and writes them to the sort buffer (the count and
    position tables, chunks x nx entries, are left out).
    - every_step: K sorts from the state of the timed steps, a re-sort
      before every full pass (the first sort sees the lattice order, the
      others the previous sort's order moved by one step);
    - random_order: one sort of a randomly permuted copy of that state (the
      first re-sort after a permutation; the passes before and after it are
      not counted), median of three permutations."""
    tpb, bpsm, resort = launch
    es = 4 if sim.precision == 32 else 8
    bytes_per_sort = (es * (5 if sim.decorated else 3) * 2 + es) * n
    peak, peak_src = measured_peak()

    def sort_span(k_steps):
        swpic.swpic_set_launch(sim.ctx, tpb, bpsm, 1)
        swpic.swpic_set_timing(sim.ctx, 1)
        torch.cuda.synchronize()
        l0 = swpic.swpic_launch_count(sim.ctx)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        # keep the stream busy (~2 ms) while the call is enqueued, so that no
        # host-side launch latency lands between the events
        with torch.cuda.stream(sim.stream):
            torch.cuda._sleep(4_000_000)
        e0.record(sim.stream)
        sim.step(k_steps, args.diag_every)
        e1.record(sim.stream)
        e1.synchronize()
        total = e0.elapsed_time(e1)
        pass_ms = swpic.swpic_pass_times(sim.ctx)
        launches = swpic.swpic_launch_count(sim.ctx) - l0
        swpic.swpic_set_timing(sim.ctx, 0)
        swpic.swpic_set_launch(sim.ctx, tpb, bpsm, resort)
        sorts, rem = divmod(launches - len(pass_ms), 5)      # 5 launches per sort
        if rem or sorts <= 0:
            raise RuntimeError("sort leg: %d launches for %d passes" % (launches, len(pass_ms)))
        return (total - float(np.sum(pass_ms))) / sorts, sorts

    def entry(ms, sorts):
        gbs = bytes_per_sort / (ms / 1e3) / 1e9
        return {"ms_per_sort": ms, "sorts": sorts, "particles_per_s": n / (ms / 1e3),
                "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                             "frac": gbs / peak, "traffic": None, "peak_source": peak_src,
                             "algorithmic_bytes_per_launch": bytes_per_sort}}

    restore(sim)
    sim.step(args.warmup, args.diag_every)
    k = max(3, min(args.steps, 20))
    ms_in, sorts_in = sort_span(k)
    rand = []
    for rep in range(3):
        restore(sim)
        sim.step(args.warmup, args.diag_every)
        g = torch.Generator(device=sim.Q.device)
        g.manual_seed(20260 + rep)
        perm = torch.randperm(n, device=sim.Q.device, generator=g)
        torch.cuda.synchronize()
        for t in arrays(sim):
            t.copy_(t[perm])
        torch.cuda.synchronize()
        swpic.swpic_refresh(sim.ctx)
        rand.append(sort_span(2))     # passes at steps 0, 1 and the closing one; one sort before step 1
    restore(sim)
    ms_r = float(np.median([r[0] for r in rand]))
    return {"kernels": "k_sort_hist, k_scan_reduce, k_scan_top, k_scan_down, k_sort_scatter",
            "bytes_per_particle": bytes_per_sort // n,
            "every_step": entry(ms_in, sorts_in), "random_order": entry(ms_r, 1),
            "note": "sort time = device time of the call minus its timed passes, per sort; "
                    "every_step: K sorts from the state of the timed steps, a re-sort before every "
                    "full pass (the first sees the lattice order, the others the previous sort's "
                    "order moved by one step); random_order: one sort of a randomly permuted state; "
                    "traffic null (the ncu summary covers the first sort on a smaller lattice)"}


def kmeans_leg(torch, swpic):
    """Decorated particles from 1e5 two-stream markers in 1e4 k-means clusters
    (10 Lloyd iterations + lumping) through swpic_kmeans_lump, device-timed;
    the FP64/FP32 oracle on a bounded sample (2e4 markers, 1e3 clusters)."""
    M, K, iters = 100000, 10000, 10
    m = W.two_stream_markers(M, 7)
    dev = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=dt)
    Qm, Pm, wm = dev(m["Q"]), dev(m["P"]), dev(m["psi"])
    outs = [torch.zeros(K, dtype=torch.float64, device="cuda") for _ in range(5)]
    assign = torch.zeros(M, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    L = 2 * np.pi

    def call():
        cq, cp = dev(m["Q"][:K]), dev(m["P"][:K])
        return swpic.swpic_kmeans_lump(Qm.data_ptr(), Pm.data_ptr(), wm.data_ptr(), M, cq.data_ptr(),
                                       cp.data_ptr(), K, L, iters, assign.data_ptr(),
                                       *[o.data_ptr() for o in outs], stream.cuda_stream)
    call()
    best = 1e30
    n = 0
    for _ in range(3):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n = call()
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    evals = M * K * (iters + 1)
    return {"markers": M, "clusters": K, "iterations": iters, "decorated_particles": int(n),
            "gpu_ms": best, "center_distance_evals_per_s": evals / (best / 1e3),
            "note": "the oracle's rate on a bounded sample is in cpu_baseline.init_kmeans"}


def p2_leg(torch, swpic, spec, args, launch, timed):
    """The same workload with the field in quadratic Lagrange elements (Sec. 5,
    k = 2), device-timed like the main line; then the energy behaviour of the
    P1 field with each phi'' projection and of the P2 field over warm-up + K
    steps from t = 0 (Hamiltonian sampled every 10 steps)."""
    lat = spec.lattice
    n = lat.n
    tpb, bpsm, resort, stages = launch
    tuned = False

    def make(d2, cap):
        s = swpic.Simulation([(lat.L, spec.dt, spec.nx, n)], precision=32, d2_mode=d2,
                             resort_every=max(resort, 0), diag_capacity=cap)
        swpic.swpic_set_launch(s.ctx, tpb, bpsm, resort)
        swpic.swpic_set_pipeline(s.ctx, stages)
        s.init_lattice(0, lat)
        swpic.swpic_refresh(s.ctx)
        return s

    if args.resort < 0 and not args.no_autotune and args.launch is None and args.stages is None:
        # P2 adds one shared atomic per particle: tune its own launch shape and
        # resort cadence on the state the timed region starts from
        s = make(swpic.SWPIC_D2_P2, 64)
        s.step(args.warmup, args.diag_every)
        swpic.swpic_autotune(s.ctx, max(5, min(args.steps, 50)), None)
        tpb, bpsm, resort = swpic.swpic_get_launch(s.ctx)
        stages = swpic.swpic_get_pipeline(s.ctx)[1]
        s.close()
        tuned = True
    s = make(swpic.SWPIC_D2_P2, 64)
    s.step(args.warmup, args.diag_every)
    ms = timed(s, args.steps)
    s.close()
    # per-pass device durations over the same warm-up + K steps from t = 0
    s = make(swpic.SWPIC_D2_P2, 64)
    s.step(args.warmup, args.diag_every)
    swpic.swpic_set_timing(s.ctx, 1)
    s.step(args.steps, args.diag_every)
    pass_ms = swpic.swpic_pass_times(s.ctx)
    s.close()
    avg_pass_ms = float(np.mean(pass_ms[1:-1] if len(pass_ms) > 2 else pass_ms))
    bpp = BYTES_PER_PARTICLE[(32, True)]
    peak, peak_src = measured_peak()
    achieved = bpp * n / (avg_pass_ms / 1e3) / 1e9
    every, total = 10, args.warmup + args.steps
    energy = {}
    for d2, name in ((swpic.SWPIC_D2_LUMPED, "p1_lumped"), (swpic.SWPIC_D2_NODAL, "p1_nodal"),
                     (swpic.SWPIC_D2_P2, "p2")):
        s = make(d2, total // every + 8)
        s.step(total, every)
        d = s.diagnostics()
        s.close()
        H, Wf = d[:, 5], d[:, 4]
        energy[name] = {"max_abs_dH": float(np.max(np.abs(H - H[0]))),
                        "max_abs_dH_over_H0": float(np.max(np.abs(H - H[0])) / abs(H[0])),
                        "max_abs_dH_over_max_W": float(np.max(np.abs(H - H[0])) / np.max(Wf)),
                        "W_final_over_W0": float(Wf[-1] / Wf[0])}
    return {"value": n * args.steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "d2_mode": "P2",
            "launch": {"threads_per_block": tpb, "blocks_per_sm": bpsm, "bulk_copy_stages": stages,
                       "resort_every": resort, "autotuned": tuned},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": profiled_traffic("k_pass_p2_bump_on_tail_4096"),
                         "avg_launch_ms": avg_pass_ms,
                         "kernel": "k_pass<float, decorated, atomic, deposit, diag, P2>",
                         "algorithmic_bytes_per_launch": bpp * n, "peak_source": peak_src},
            "energy_behaviour": energy, "energy_steps": total, "energy_sample_every": every,
            "note": "the oracle's P2 rate on a bounded sample is in cpu_baseline.p2_elements"}


BYTES_PER_PARTICLE_2D = {32: 68, 64: 136}     # read Q, P, q*, p* (2 each) and psi*; write all but psi*


def two_d_leg(torch, swpic, args):
    """The 2D2V step (general-d model of Sec. 3.3 on the torus, bilinear
    elements): oblique Landau damping, k = (1/2, 1/2) on [0, 4 pi)^2,
    alpha 0.05, a side^4 decorated lattice (64^4 = 16,777,216 FP32 particles,
    built on the device) on a 32 x 32 mesh, dt 0.05, diagnostics every step;
    warm-up W steps, K device-timed steps, then the per-pass roofline over
    steps restarted from the lattice.  The dipole weights grow in time (the
    shear of nearby characteristics), so no part runs past t = (W + K) dt."""
    side = int(round(args.side_2d ** 0.5))
    spec = W.landau_2d(side)
    n, L, nx, dt = spec.n, spec.Lx, 32, 0.05
    sim = swpic.Simulation2D(L, L, nx, nx, dt, n, precision=32, diag_capacity=args.warmup + 2 * args.steps + 8)
    try:
        sim.init_lattice(spec)
        sim.step(args.warmup, args.diag_every)
        swpic.swpic2d_synchronize(sim.ctx)
        l0 = swpic.swpic2d_launch_count(sim.ctx)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.step(args.steps, args.diag_every)
        e1.record(sim.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        launches = swpic.swpic2d_launch_count(sim.ctx) - l0
        d = sim.diagnostics()
        # end to end through swpic2d_step_host on the same segment: pinned host
        # state after the W warm-up steps in, the K steps, the state out
        sim.init_lattice(spec)
        sim.step(args.warmup, args.diag_every)
        st = sim.state()
        keys = swpic.STATE2D
        hin = [torch.from_numpy(st[k].astype(np.float32)).pin_memory() for k in keys]
        hout = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in keys[:8]]
        del st
        swpic.swpic2d_step_host(sim.ctx, [t.data_ptr() for t in hin], [t.data_ptr() for t in hout], 3,
                                args.diag_every)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        swpic.swpic2d_step_host(sim.ctx, [t.data_ptr() for t in hin], [t.data_ptr() for t in hout], args.steps,
                                args.diag_every)
        e2e_s = time.perf_counter() - t0
        del hin, hout
        sim.init_lattice(spec)
        sim.step(args.warmup, args.diag_every)
        swpic.swpic2d_set_timing(sim.ctx, 1)
        sim.step(min(args.steps, 200), args.diag_every)
        pass_ms = swpic.swpic2d_pass_times(sim.ctx)
        swpic.swpic2d_set_timing(sim.ctx, 0)
    finally:
        sim.close()
    full = pass_ms[1:-1] if len(pass_ms) > 2 else pass_ms
    avg = float(np.mean(full))
    bpp = BYTES_PER_PARTICLE_2D[32]
    peak, peak_src = measured_peak()
    achieved = bpp * n / (avg / 1e3) / 1e9
    H = d[:, 6]
    d = d[: args.warmup + args.steps + 1] if args.diag_every == 1 else d
    return {"workload": "landau2d_oblique_lattice_%d^4_mesh_32x32" % side, "particles": n, "mesh": [nx, nx], "dt": dt,
            "value": n * args.steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "gpu_launches": int(launches),
            "e2e": {"value": n * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 36 * n / args.steps,
                    "d2h_bytes_per_step": 32 * n / args.steps,
                    "note": "swpic2d_step_host on the state after the W warm-up steps: H2D of the 9 arrays, "
                            "field set-up, K steps, D2H of 8 arrays, all inside the timed region"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "avg_launch_ms": avg,
                         "traffic": profiled_traffic("k_pass2d_landau2d_64x64x64x64") if n == 1 << 24 else None,
                         "kernel": "k_pass2d<float, decorated, deposit, diag>",
                         "algorithmic_bytes_per_launch": bpp * n, "peak_source": peak_src},
            "max_abs_dH_over_H0": float(np.max(np.abs(H - H[0])) / abs(H[0])),
            "note": "the oracle's 2D rate on a bounded sample is in cpu_baseline.two_d"}


def ensemble_leg(torch, swpic):
    """256 independent Landau runs (uneven lattices 64^2..512^2, nx = side/2,
    800 steps, diagnostics every step): one graph-captured batched context vs
    the same runs one after another with plain launches.  Equal error: the
    fitted damping rate of the linear runs (alpha < 0.05) against the kinetic
    dispersion root."""
    from workloads import physics as ph
    runs = W.ensemble(precision=32)
    steps = runs[0].steps

    def run_batched():
        sim = swpic.Simulation([(r.lattice.L, r.dt, r.nx, r.lattice.n) for r in runs], precision=32,
                               diag_capacity=steps + 8)
        for i, r in enumerate(runs):
            sim.init_lattice(i, r.lattice)
        swpic.swpic_refresh(sim.ctx)
        swpic.swpic_synchronize(sim.ctx)
        t0 = time.perf_counter()
        sim.step(steps, 1)
        sync_tolerant(sim.ctx)
        dt = time.perf_counter() - t0
        flags = swpic.swpic_run_status(sim.ctx, len(runs))
        diags = [sim.diagnostics(i) for i in range(len(runs))]
        sim.close()
        return dt, diags, flags

    def run_plain():
        sims = []
        for r in runs:
            s = swpic.Simulation([(r.lattice.L, r.dt, r.nx, r.lattice.n)], precision=32,
                                 use_graphs=False, diag_capacity=steps + 8, with_scratch=False)
            s.init_lattice(0, r.lattice)
            swpic.swpic_refresh(s.ctx)
            sims.append(s)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in sims:
            s.step(steps, 1)
            sync_tolerant(s.ctx)
        dt = time.perf_counter() - t0
        flags = np.array([swpic.swpic_run_status(s.ctx, 1)[0] for s in sims])
        diags = [s.diagnostics() for s in sims]
        for s in sims:
            s.close()
        return dt, diags, flags

    def sync_tolerant(ctx):
        # runs whose decorations blow up (nonlinear runs late in time) flag a
        # fixed-point overflow; they are counted, the others are unaffected
        try:
            swpic.swpic_synchronize(ctx)
        except swpic.SwpicError as e:
            if e.status != swpic.SWPIC_ENUMERIC:
                raise

    def gamma_err(diags):
        """Per run: the damping rate fitted over t in [2, t1], t1 = min(0.8 T_R,
        2/|gamma_root|, 40) (at least 12): before the lattice recurrence T_R =
        2 pi/(k dv), over about two e-folds of the damping, and before the
        nonlinear trapping time of the larger alphas.  Median relative error
        against the dispersion root over the runs with alpha < 0.05, by lattice
        side, and over the resolved linear runs (side >= 256, alpha < 0.02)."""
        errs = []
        for r, d in zip(runs, diags):
            lat = r.lattice
            if lat.alpha >= 0.05:
                continue
            root = ph.landau_root(lat.kx, 1.0 + 0.5 * lat.kx - 0.1j)
            t_rec = 2 * np.pi / (lat.kx * (lat.vmax - lat.vmin) / lat.nv)
            t1 = max(12.0, min(0.8 * t_rec, 2.0 / abs(root.imag), 40.0))
            try:
                g, _, _ = ph.rate_fit(d[:, 0], d[:, 6], 2.0, t1, min_sep=1.2)
            except ValueError:
                continue
            errs.append((lat.nq, lat.alpha, abs(g / root.imag - 1)))
        med = lambda xs: float(np.median(xs)) if xs else None
        return {"median_alpha_lt_0.05": med([e for _, _, e in errs]), "runs_fitted": len(errs),
                "median_by_side": {str(sd): med([e for s_, _, e in errs if s_ == sd]) for sd in (64, 128, 256, 512)},
                "median_side_ge_256_alpha_lt_0.02": med([e for s_, a_, e in errs if s_ >= 256 and a_ < 0.02]),
                "runs_side_ge_256_alpha_lt_0.02": sum(1 for s_, a_, _ in errs if s_ >= 256 and a_ < 0.02)}

    tb, db, fb = run_batched()
    tp, dp, fp = run_plain()
    eb = gamma_err(db)
    ep = gamma_err(dp)
    total = sum(r.lattice.n for r in runs)
    return {"runs": len(runs), "particles": total, "steps": steps,
            "batched_s": tb, "plain_s": tp, "speedup": tp / tb,
            "batched_value": total * steps / tb, "plain_value": total * steps / tp,
            "gamma_rel_err_median_batched": eb["median_alpha_lt_0.05"],
            "gamma_rel_err_median_plain": ep["median_alpha_lt_0.05"],
            "gamma_rel_err_batched": eb, "gamma_rel_err_plain": ep,
            "runs_fitted": eb["runs_fitted"],
            "runs_flagged_batched": int(np.count_nonzero(fb)),
            "runs_flagged_plain": int(np.count_nonzero(fp)),
            "note": "wall time of the step calls only; equal error = same median |gamma/gamma_root - 1|"}


def device_leg(torch, swpic, spec, args, timed, tune=True):
    """One workload from the lattice start on the device: launch shape tuned on
    the state after the W warm-up steps (the autotuner restores that state),
    then K device-timed steps, and the mean device duration of the full passes
    of the same K steps for the roofline."""
    lat = spec.lattice
    n, prec, dec = lat.n, spec.precision, spec.decorated
    jx, jv = W.jitter(lat) if lat.jitter else (None, None)
    s = swpic.Simulation([(lat.L, spec.dt, spec.nx, n)], precision=prec, decorated=dec,
                         diag_capacity=64)
    try:
        s.init_lattice(0, lat, jx, jv)
        swpic.swpic_refresh(s.ctx)
        s.step(args.warmup, args.diag_every)
        if tune:
            swpic.swpic_autotune(s.ctx, 10, None)
        tpb, bpsm, resort = swpic.swpic_get_launch(s.ctx)
        stages = swpic.swpic_get_pipeline(s.ctx)[1]
        ms = timed(s, args.steps)
        s.init_lattice(0, lat, jx, jv)
        swpic.swpic_refresh(s.ctx)
        s.step(args.warmup, args.diag_every)
        swpic.swpic_set_timing(s.ctx, 1)
        s.step(args.steps, args.diag_every)
        pass_ms = swpic.swpic_pass_times(s.ctx)
        swpic.swpic_set_timing(s.ctx, 0)
    finally:
        s.close()
    avg = float(np.mean(pass_ms[1:-1] if len(pass_ms) > 2 else pass_ms))
    bpp = BYTES_PER_PARTICLE[(prec, dec)]
    peak, peak_src = measured_peak()
    achieved = bpp * n / (avg / 1e3) / 1e9
    kernel = "k_pass<%s, %s, atomic, deposit, diag>" % ("float" if prec == 32 else "double",
                                                       "decorated" if dec else "point")
    prof = {(32, False, 8192 * 8192): "k_pass_pic_landau_strong_8192"}.get((prec, dec, n))
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "avg_launch_ms": avg, "algorithmic_bytes_per_launch": bpp * n,
            "traffic": profiled_traffic(prof) if prof else None, "kernel": kernel, "peak_source": peak_src}
    if prec == 64:
        # the FP64 step is bound by the FP64 pipe, not by HBM: its arithmetic
        # (FMA = 2 flops) per particle-step against the nominal FP64 rate
        flops = FP64_FLOPS_PER_PARTICLE[dec]
        gf = flops * n / (avg / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": gf, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": gf / FP64_NOMINAL_TFLOPS, "flops_per_particle": flops, "avg_launch_ms": avg,
                "kernel": kernel, "peak_source": "nominal GB300 FP64 rate (no measured FP64 peak)",
                "hbm_achieved_gbs": achieved, "hbm_frac": achieved / peak,
                "note": "ncu on the 2048^2 lattice: the FP64 pipe is busy 83% of active cycles "
                        "(it also executes the comparisons, clamps and directed-rounding adds that "
                        "are not counted as flops); DRAM at 9%"}
    return {"workload": spec.name, "particles": n, "precision": "fp%d" % prec, "decorated": dec,
            "value": n * args.steps / (ms / 1e3), "unit": UNIT if dec else "particle-steps/s",
            "ms_per_step": ms / args.steps,
            "launch": {"threads_per_block": tpb, "blocks_per_sm": bpsm, "bulk_copy_stages": stages,
                       "resort_every": resort},
            "roofline": roof}


def method_legs(torch, swpic, args, timed):
    """Strong Landau damping (alpha 0.5, k 0.5, 2048^2 lattice with +-0.25 cell
    jitter, nx 512, dt 0.05): the decorated step in FP32 and in FP64, and the
    point-particle step (decoration off, same kernels) at 16x the particles
    (8192^2 lattice), each device-timed from the lattice start.  Then the
    comparison at equal accuracy over t in [0, 15] (300 steps): decorated and
    point-particle runs of the same problem at several lattice sizes, each
    E_amp history against the FP64 oracle's decorated run of the 2048^2
    lattice (relative RMS difference), beside the device time each run needs
    to reach t = 15, and for each error level the fewest particles with which
    each method reaches it."""
    import oracle as O
    from workloads import physics as ph
    out = {"fp32_decorated": device_leg(torch, swpic, W.landau_strong(32), args, timed),
           "fp64_decorated": device_leg(torch, swpic, W.landau_strong(64), args, timed),
           "pic_16x": device_leg(torch, swpic, W.landau_strong(32, scale=4, decorated=False), args, timed)}
    steps, t_end = 300, 15.0

    def gpu_history(sp):
        lat = sp.lattice
        jx, jv = W.jitter(lat) if lat.jitter else (None, None)
        s = swpic.Simulation([(lat.L, sp.dt, sp.nx, lat.n)], precision=sp.precision,
                             decorated=sp.decorated, diag_capacity=steps + 8)
        try:
            s.init_lattice(0, lat, jx, jv)
            swpic.swpic_refresh(s.ctx)
            s.step(steps, 1)          # warm (graphs captured, clocks up)
            s.init_lattice(0, lat, jx, jv)
            swpic.swpic_refresh(s.ctx)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
            s.step(steps, 1)
            e1.record(s.stream)
            e1.synchronize()
            d = s.diagnostics()
        finally:
            s.close()
        return d, e0.elapsed_time(e1)

    def at_side(side, dec):
        import dataclasses
        base = W.landau_strong(32, decorated=dec)
        return dataclasses.replace(base, lattice=dataclasses.replace(base.lattice, nq=side, nv=side),
                                   name="landau_strong_%dx%d%s" % (side, side, "" if dec else "_pic"))

    spec = W.landau_strong(64)
    lat = spec.lattice
    jx, jv = W.jitter(lat)
    O.set_threads(host_cores())
    try:
        t0 = time.perf_counter()
        ref = O.run(O.init_lattice(lat, jx, jv), spec.nx, lat.L, spec.dt, steps, diag_every=1)["diag"]
        t_oracle = time.perf_counter() - t0
    finally:
        O.set_threads(1)
    E_ref = ref[:, 6]
    g_ref = ph.rate_fit(ref[:, 0], E_ref, 0.0, t_end, min_sep=1.0)[0]
    rows = []
    for dec, sides in ((True, (256, 512, 1024, 2048)), (False, (256, 512, 1024, 2048, 4096, 8192))):
        for side in sides:
            sp = at_side(side, dec)
            d, ms = gpu_history(sp)
            E = d[: len(E_ref), 6]
            ok = bool(np.all(np.isfinite(E)))
            err = float(np.sqrt(np.mean((E - E_ref) ** 2) / np.mean(E_ref ** 2))) if ok else None
            rows.append({"method": "decorated" if dec else "point", "lattice": side,
                         "particles": side * side, "device_ms_to_t15": ms, "finite": ok,
                         "E_amp_rel_rms_err": err})

    def cheapest(method, tol):
        c = [r for r in rows if r["method"] == method and r["finite"] and r["E_amp_rel_rms_err"] <= tol]
        return min(c, key=lambda r: r["particles"]) if c else None
    equal = {}
    for tol in (1e-2, 1e-3, 1e-4):
        a, b = cheapest("decorated", tol), cheapest("point", tol)
        equal["%g" % tol] = {"decorated": None if a is None else {k: a[k] for k in ("particles", "device_ms_to_t15")},
                             "point": None if b is None else {k: b[k] for k in ("particles", "device_ms_to_t15")}}
    out["equal_accuracy"] = {
        "window": [0.0, t_end], "steps": steps,
        "reference": "FP64 oracle, decorated, 2048^2 lattice (%d particles), particle loops on %d host "
                     "threads, %.1f s" % (lat.n, host_cores(), t_oracle),
        "gamma_fit_reference": float(g_ref),
        "error": "relative RMS difference of the E_amp history over the window from the reference",
        "runs": rows,
        "fewest_particles_within": equal,
        "note": "GPU FP32 runs of the same problem (alpha 0.5, k 0.5, +-0.25 cell jitter, nx 512, "
                "dt 0.05) at several lattice sizes, with and without decorations"}
    return out


def fp32_diag_error_leg(torch, swpic, spec, args):
    """The error of every diagnostic of the FP32 step against the FP64 oracle
    started from the same (FP32-representable) state: two-stream (256^2,
    600 steps to t = 30, records every 10 steps) and the bump-on-tail
    workload (4096^2, W + K steps from the lattice start, records every
    step).  The error of a quantity is max over records |FP32 - FP64| over
    its largest FP64 magnitude; the momentum, which stays near zero, is
    measured against mass x v_rms = (2 mass kinetic)^(1/2) instead."""
    import oracle as O
    keys = ["mass", "momentum", "kinetic", "field_energy", "H", "E_amp"]

    def compare(sp, steps, every, threads):
        lat = sp.lattice
        st0 = O.init_lattice(lat)
        st = {k: v.astype(np.float32).astype(np.float64) for k, v in st0.items()}
        del st0
        s = swpic.Simulation([(lat.L, sp.dt, sp.nx, lat.n)], precision=32, diag_capacity=steps // every + 8)
        try:
            s.init_particles(st)
            s.step(steps, every)
            g = s.diagnostics()
        finally:
            s.close()
        O.set_threads(threads)
        try:
            o = O.run(st, sp.nx, lat.L, sp.dt, steps, diag_every=every)["diag"]
        finally:
            O.set_threads(1)
        err = {}
        for i, k in enumerate(keys):
            a, b = g[: len(o), i + 1], o[:, i + 1]
            scale = np.max(np.abs(b))
            if k == "momentum":
                scale = float(np.sqrt(2 * o[0, 1] * o[0, 3]))
            err[k] = float(np.max(np.abs(a - b)) / scale)
        return {"workload": sp.name, "particles": lat.n, "steps": steps, "record_every": every,
                "rel_error": err}

    return {"two_stream": compare(W.two_stream(32), 600, 10, 1),
            "bump_on_tail": compare(spec, args.warmup + args.steps, 1, host_cores()),
            "note": "FP32 state and push, FP64 field energy; errors relative to each quantity's "
                    "largest FP64 value (momentum: to (2 mass kinetic)^(1/2))"}


def cpu_baseline_leg(spec, args):
    """The FP64 oracle on the host cores: all of them (particle loops split
    into blocks, or_set_threads) and one, on the same bounded sample."""
    cols = 256                     # 256 x 4096 = 1,048,576 particles
    k = 20
    n, dt, cores, m = time_oracle(spec, cols, k, 0, args.diag_every, threads=host_cores())
    n1, dt1, _, m1 = time_oracle(spec, cols, 5, 0, args.diag_every, threads=1)
    how = ("%d of %d lattice columns (%d particles) of %s from the lattice start, plain-C FP64 "
           "oracle; seconds per step = [t(M+1 steps) - t(1 step)]/M, each the best of two runs "
           "(the one-time dense LU of each oracle run left out)" % (cols, spec.lattice.nq, n, spec.name))
    return {"value": n * k / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": how + ", M = %d, particle loops on %d host threads" % (m, cores),
            "host_cores": host_cores(),
            "single_core": {"value": n1 * 5 / dt1, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": how + ", M = %d, serial loops" % m1},
            "init_kmeans": kmeans_oracle_sample(), "p2_elements": p2_oracle_sample(spec, args),
            "two_d": two_d_oracle_sample(args)}


def two_d_oracle_sample(args):
    """The 2D oracle on a 16^4 lattice (65,536 particles) of the 2D workload's
    f0 (same domain, mesh and dt), 5 steps, one core (its dense LU of the
    1025 x 1025 bordered system is included)."""
    import oracle as O
    spec = W.landau_2d(16)
    st = O.init_lattice2d(spec)
    k = 5
    t0 = time.perf_counter()
    O.run2d(st, 32, 32, spec.Lx, spec.Ly, 0.05, k, diag_every=args.diag_every)
    t = time.perf_counter() - t0
    return {"value": spec.n * k / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "16^4 lattice (%d particles) of the 2D workload's f0, 32 x 32 mesh, %d steps" % (spec.n, k)}


def p2_oracle_sample(spec, args):
    """The oracle with the P2 field (a dense (2 nx + 1)^2 LU solve every step)
    on 64 lattice columns, 3 steps, one core."""
    cols, k = 64, 3
    n, dt, _, _ = time_oracle(spec, cols, k, 0, args.diag_every, 3)
    return {"value": n * k / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d of %d lattice columns (%d particles), %d steps, P2 field" %
                      (cols, spec.lattice.nq, n, k)}


def kmeans_oracle_sample():
    """The oracle's k-means initialization on a bounded sample: 2e4 two-stream
    markers, 1e3 clusters, 8 Lloyd iterations + lumping, one core."""
    import oracle as O
    Ms, Ks, its, L = 20000, 1000, 8, 2 * np.pi
    m = W.two_stream_markers(Ms, 1)
    t0 = time.perf_counter()
    cq, cp, a = O.kmeans(m["Q"], m["P"], m["psi"], m["Q"][:Ks], m["P"][:Ks], L, its)
    O.lump(m["Q"], m["P"], m["psi"], a, cq, cp, L)
    t = time.perf_counter() - t0
    return {"markers": Ms, "clusters": Ks, "iterations": its, "seconds": t, "cores": 1,
            "center_distance_evals_per_s": Ms * Ks * (its + 1) / t}


if __name__ == "__main__":
    main()
