"""Benchmark: aggregate walker-ns/day and pair interactions/s of the batched
multiple-walker lambda-ABF step on the solvation-like workload (4096
flexible 3-site waters + a 12-site neutral alchemical solute, 12 300 atoms,
5 nm box, reaction field, r_c = 1.0 nm, 16 walkers in a vdW and a Coulomb
stage of 100 bins each, 1 fs steps), synthetic seeded inputs.

One bench step = one la_step_walkers call advancing every walker by
--md-steps MD steps (each MD step runs every part of the path: BAOAB of
atoms and lambda, neighbour-list rebuild when needed, pair forces with
dU/dlambda, bonded terms, ABF fold and bias).  L2 is flushed between bench
steps (a 256 MB write).  `value` is timed with CUDA events on the engine's
stream with the state resident in HBM; `e2e` times the same work through
the C ABI with the walker state uploaded from pinned host memory before and
read back (state + ABF accumulators) after every bench step.

--impl reference times the FP64 oracle (the plain CPU statement of the
method) on this machine's host cores on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "aggregate walker-ns/day"
UNIT = "walker-ns/day"
FLOP_PER_PAIR = 37  # FP32 flops per in-cutoff LJ+RF pair, force only (FMA = 2); see k_pairs.cu
SKIN_NM = 0.15  # list radius r_c + skin
PRUNE_NM = 0.06  # pair-pass pruning margin (0: off); measured best with SKIN_NM


def workload_name(skin=SKIN_NM, prune=PRUNE_NM):
    return ("solvation-like: 4096 flexible 3-site waters + 12-site alchemical solute "
            f"(12300 atoms, 5 nm box, RF eps_rf=78, r_c=1.0 nm, list skin {skin:g} nm, "
            f"pruning margin {prune:g} nm), 16 walkers "
            "(8 vdW-stage on [0,0.5] + 8 Coulomb-stage on [0.5,1]), 100 bins per stage, dt=1 fs, 300 K")




def workload(skin=SKIN_NM):
    from paper_2307_08006_gb300 import synth

    spec = synth.water_box(4096, 12, seed=8007)
    run = synth.water_run(seed=8007, walkers_per_stage=8, n_bins=100, n_full=200.0, skin=skin)
    return spec, run


def walker_ns_per_day(n_walkers, md_steps, dt_ps, seconds):
    return n_walkers * md_steps * dt_ps * 1e-3 / seconds * 86400.0


# ---------------------------------------------------------------------------
def cpu_baseline(steps=2, single_thread=False):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of
    the same workload (all 16 walkers, `steps` MD steps, OpenMP over walkers)."""
    import oracle

    spec, run = workload()
    from paper_2307_08006_gb300 import synth

    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    st = synth.initial_state(spec, run)
    sim = oracle.Simulation(spec, run, st)  # includes one force evaluation (untimed)
    t0 = time.perf_counter()
    sim.run(steps)
    dt = time.perf_counter() - t0
    val = walker_ns_per_day(run.n_walkers, steps, run.dt, dt)
    out = dict(value=val, unit=UNIT, cores=cores, kind="oracle",
               sample=f"{run.n_walkers} walkers x {steps} MD steps of the same workload "
                      f"(O(N^2) FP64, OpenMP over walkers), {dt:.2f} s")
    if single_thread:
        # the same oracle on one core: one walker of each stage, one MD step
        from dataclasses import replace

        run1 = replace(run, stages=[replace(s_, n_walkers=1) for s_ in run.stages])
        oracle.set_threads(1)
        sim1 = oracle.Simulation(spec, run1, synth.initial_state(spec, run1))
        t1 = time.perf_counter()
        sim1.run(1)
        d1 = time.perf_counter() - t1
        oracle.set_threads(cores)
        out["single_thread"] = dict(value=walker_ns_per_day(run1.n_walkers, 1, run.dt, d1), unit=UNIT, cores=1,
                                    sample=f"{run1.n_walkers} walkers x 1 MD step, one thread, {d1:.2f} s")
    return out, dt


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    steps_total, secs_total = 0, 0.0
    cb = None
    for k in range(args.warmup + args.steps):
        cbk, dt = cpu_baseline(steps=1)
        if k >= args.warmup:
            steps_total += 1
            secs_total += dt
            cb = cbk
    spec, run = workload(args.skin)
    val = walker_ns_per_day(run.n_walkers, steps_total, run.dt, secs_total)
    cb["value"] = val
    line = dict(impl="reference", metric=METRIC, value=val, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * secs_total / max(steps_total, 1),
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=workload_name(args.skin, args.prune_margin), walkers=run.n_walkers,
                            atoms_per_walker=spec.n, md_steps_per_bench_step=1),
                cpu_baseline=cb, e2e=dict(value=val, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, dev_index=0):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["unavailable"])
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9 and r[0].strip() == str(dev_index)]
        if not rows:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["unavailable"])
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=reasons, samples=len(rows))


def measured_traffic(variant):
    """DRAM bytes per pair-kernel launch from the committed ncu summary, or
    None when the capture is of older kernel source.  The fused step launch
    is preferred; otherwise the one-task launch of the same variant."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "k_pairs_solvation16.md")
    try:
        text = open(path).read()
    except OSError:
        return None, "no capture"
    lines = re.findall(r"traffic_bytes_per_launch: variant=(\d+) form=(\w+) dram_bytes=(\d+) "
                       r"source_sha256=(\w+)", text)
    if not lines:
        return None, "no capture"
    h = hashlib.sha256()
    for f in ("k_pairs.cu", "labf_internal.cuh", "labf_dyn.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2307_08006_gb300", "csrc", f), "rb").read())
    if h.hexdigest()[:16] != lines[0][3]:
        return None, "kernel source changed since the capture"
    for form in ("fused", "single"):
        for v, fm, b, _ in lines:
            if int(v) == variant and fm == form:
                return int(b), f"profiles/k_pairs_solvation16.md (ncu, {form} launch, variant {v})"
    return None, f"no capture of pair_variant={variant}"


def measured_hbm():
    """HBM copy bandwidth measured on this machine (GB/s), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def flush_l2(buf):
    buf.add_(1)  # 256 MB read + write, larger than the 129 MB L2


def _timed_steps(eng, md_steps, stream, plain=False):
    """Device milliseconds of md_steps MD steps (CUDA events on the stream)."""
    import torch

    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    (eng.step_plain if plain else eng.step)(md_steps, stream)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def _count_pairs(eng):
    n = a = 0
    for w in range(eng.n_walkers):
        r = eng.energy_forces(w, count_pairs=True, forces=False)
        n += r["pairs_normal"]
        a += r["pairs_alch"]
    return n, a


def bench_uneven(args, stream, peak_tflops):
    """Batched uneven systems: 64 walkers over 8 water boxes of 256 ... 8192
    waters (4 ... 40-site solutes), one graph, autotuned, against one launch
    sequence per walker without graphs on the same GPU."""
    from paper_2307_08006_gb300 import labf, synth

    inputs = []
    for k, sp in enumerate(synth.uneven_batch(8008)):
        rng = np.random.default_rng(8008 + k)
        sp.x = ((sp.x + rng.normal(0.0, 0.01, sp.x.shape)) % sp.box).astype(np.float32)
        run = synth.uneven_run(seed=8008 + k, walkers_per_system=8)
        # the bench's list skin where the box allows it (2 (r_c + skin) <= L)
        if sp.box >= 2.0 * (sp.r_cut + args.skin):
            run.skin = args.skin
        inputs.append(labf.SystemInput(sp, run, synth.initial_state(sp, run)))
    t0 = time.perf_counter()
    eng = labf.Engine(inputs, options=dict(graph_steps=args.graph_steps, autotune=1, prune_margin=args.prune_margin))
    eng.step(args.settle // 2)
    eng.sync()
    eng.autotune()
    setup_s = time.perf_counter() - t0
    pn, pa = _count_pairs(eng)
    W = eng.n_walkers
    atoms = sum(si.spec.n * si.run.n_walkers for si in inputs)
    dt = inputs[0].run.dt
    md = args.md_steps
    _timed_steps(eng, md, stream)  # warm-up
    rb0 = int(eng.stats()[1])
    ms = sum(_timed_steps(eng, md, stream) for _ in range(3)) / 3.0
    rebuild_rate = (int(eng.stats()[1]) - rb0) / float(W * 3 * md)
    plain_md = max(5, md // 20)
    _timed_steps(eng, 2, stream, plain=True)
    pms = _timed_steps(eng, plain_md, stream, plain=True)
    kt = eng.time_kernels(args.profile_steps, stream)
    st = eng.stats()
    out = dict(
        workload="batched uneven systems: 8 water boxes (256, 512, 1024, 2048, 3072, 4096, 6144, 8192 waters; "
                 "4-40-site alchemical solutes; r_c 1.0 nm, 0.85 nm for the 1.98 nm box; list skin "
                 f"{args.skin:g} nm, 0.1 nm for the 1.98 nm box; pruning margin {args.prune_margin:g} nm), "
                 "8 walkers each (64), one CUDA graph, autotuned",
        walkers=W, atoms_all_walkers=atoms, md_steps=3 * md,
        value=walker_ns_per_day(W, md, dt, ms * 1e-3), unit=UNIT, ms_per_md_step=ms / md,
        pair_interactions_per_s=(pn + pa) * md / (ms * 1e-3), in_cutoff_pairs_per_md_step=pn + pa,
        plain_form=dict(value=walker_ns_per_day(W, plain_md, dt, pms * 1e-3), unit=UNIT, md_steps=plain_md,
                        ms_per_md_step=pms / plain_md, note="one walker per launch sequence, no CUDA graph"),
        batched_over_plain=(pms / plain_md) / (ms / md),
        lists=dict(tiles_8x4=int(st[6]), cluster_pair_entries=int(st[5]),
                   tile_efficiency=pn / max(1, 32 * int(st[6])), rebuilds_per_walker_md_step=rebuild_rate),
        kernel_ms=dict((k, v[0]) for k, v in kt.items()),
        launch=eng.autotune_report(), setup_s=setup_s)
    pair_ms = kt["pairs"][0]
    ach = (pn + pa) * FLOP_PER_PAIR / (pair_ms * 1e-3) / 1e12
    out["roofline"] = dict(bound="alu", achieved=ach, peak=peak_tflops, unit="TFLOP/s", frac=ach / peak_tflops,
                           pair_kernel_ms=pair_ms)
    eng.close()
    return out


def bench_large(args, stream, peak_tflops):
    """Large synthetic complex: 31 000 waters + a 3000-site restrained chain +
    a 40-site alchemical ligand with a flat-bottom restraint (96 040 atoms,
    r_c 1.2 nm), 16 walkers."""
    from paper_2307_08006_gb300 import labf, synth

    sp = synth.large_complex()
    run = synth.large_complex_run()
    run.skin = args.skin
    t0 = time.perf_counter()
    eng = labf.Engine([labf.SystemInput(sp, run, synth.initial_state(sp, run))],
                      options=dict(graph_steps=args.graph_steps, autotune=1, prune_margin=args.prune_margin))
    eng.step(args.settle // 4)
    eng.sync()
    eng.autotune()
    setup_s = time.perf_counter() - t0
    pn, pa = _count_pairs(eng)
    W = eng.n_walkers
    md = max(20, args.md_steps // 2)
    _timed_steps(eng, md, stream)
    rb0 = int(eng.stats()[1])
    ms = sum(_timed_steps(eng, md, stream) for _ in range(3)) / 3.0
    rebuild_rate = (int(eng.stats()[1]) - rb0) / float(W * 3 * md)
    kt = eng.time_kernels(max(5, args.profile_steps // 2), stream)
    st = eng.stats()
    pair_ms = kt["pairs"][0]
    ach = (pn + pa) * FLOP_PER_PAIR / (pair_ms * 1e-3) / 1e12
    out = dict(
        workload="large synthetic complex: 31000 flexible waters + 3000-site chain (0.15 nm bonds, positional "
                 "restraints) + 40-site alchemical ligand (flat-bottom restraint to the chain), 96040 atoms, "
                 f"9.92 nm box, r_c 1.2 nm, list skin {args.skin:g} nm, pruning margin {args.prune_margin:g} nm",
        walkers=W, atoms_per_walker=sp.n, md_steps=3 * md,
        value=walker_ns_per_day(W, md, run.dt, ms * 1e-3), unit=UNIT, ms_per_md_step=ms / md,
        pair_interactions_per_s=(pn + pa) * md / (ms * 1e-3), in_cutoff_pairs_per_md_step=pn + pa,
        lists=dict(tiles_8x4=int(st[6]), cluster_pair_entries=int(st[5]),
                   tile_efficiency=pn / max(1, 32 * int(st[6])),
                   rebuilds_per_walker_md_step=rebuild_rate),
        kernel_ms=dict((k, v[0]) for k, v in kt.items()),
        roofline=dict(bound="alu", achieved=ach, peak=peak_tflops, unit="TFLOP/s", frac=ach / peak_tflops,
                      pair_kernel_ms=pair_ms,
                      kernel="k_pairs, fused step launch (normal + alchemical pairs, bonded, walker, lambda)"),
        launch=eng.autotune_report(), setup_s=setup_s)
    eng.close()
    return out


def bench_autograd(args):
    """Differentiation on the bench system (C4 shape): U and its gradients
    with respect to the positions, lambda and the solute's (epsilon, sigma,
    q) through torch.autograd, one walker, at 21 lambda values from 0 to 1.
    Every call hands the device tensors to the engine, which rebuilds the
    walker's lists from the positions and evaluates U with the hand-written
    derivative pass; nothing goes through host memory."""
    import torch

    from paper_2307_08006_gb300 import autograd, labf, synth

    spec, _ = workload(args.skin)
    run = synth.water_run(seed=8010, walkers_per_stage=1, skin=args.skin)
    run.stages = [synth.Stage(0.0, 1.0, 20, 1)]
    state = synth.initial_state(spec, run, lam0=[0.5])
    eng = labf.engine_for(spec, run, state)
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.tensor(state.x[0], device=dev, requires_grad=True)
    th = torch.tensor(autograd.theta_of(spec), dtype=torch.float64, device=dev, requires_grad=True)
    lams = [torch.tensor(k / 20.0, dtype=torch.float64, device=dev, requires_grad=True) for k in range(21)]

    def sweep():
        for lt in lams:
            U = autograd.energy(eng, 0, x, lt, th)
            torch.autograd.grad(U, [x, lt, th])

    sweep()  # warm-up
    reps = 3
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a.record()
    for _ in range(reps):
        sweep()
    b.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    n = reps * len(lams)
    eng.close()
    return dict(workload="differentiation on the bench system (12300 atoms, one walker): U and dU/dx, "
                         "dU/dlambda, dU/d(epsilon, sigma, q) of the 12 solute sites through torch.autograd "
                         "at 21 lambda values; lists rebuilt from x on every call",
                calls=n, ms_per_call=a.elapsed_time(b) / n, wall_ms_per_call=wall / n * 1e3,
                note="forward + backward per call, CUDA events on the current stream")


def gpu_arm(args):
    import torch

    from paper_2307_08006_gb300 import labf, synth

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec, run = workload(args.skin)
    state = synth.initial_state(spec, run, seed=run.seed + 1000 * rank)
    opts = dict(graph_steps=args.graph_steps, autotune=int(args.autotune), prune_margin=args.prune_margin)
    if args.launch:  # a fixed pair-kernel launch shape instead of the tuner's
        for kv in args.launch.split(","):
            k, v = kv.split("=")
            if k not in ("pair_variant", "pair_ctas_per_sm", "chunk_entries"):
                raise SystemExit(f"unknown launch option {k}")
            opts[k] = int(v)
        opts["autotune"] = 0
    eng = labf.Engine([labf.SystemInput(spec, run, state)], options=opts, device=local)
    stream = torch.cuda.current_stream(dev)
    md = args.md_steps
    # settle the lattice start (untimed): 2 ps; then tune the pair kernel on
    # the settled lists
    eng.step(args.settle)
    eng.sync()
    if args.autotune and not args.launch:
        eng.autotune()
    # in-cutoff pairs per MD step (all walkers), counted at the settled state
    pairs_n = pairs_a = 0
    for w in range(eng.n_walkers):
        r = eng.energy_forces(w, count_pairs=True, forces=False)
        pairs_n += r["pairs_normal"]
        pairs_a += r["pairs_alch"]
    pairs_per_md = pairs_n + pairs_a
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def bench_step():
        eng.step(md, stream)

    for _ in range(args.warmup):
        bench_step()
        flush_l2(flush)
    torch.cuda.synchronize()
    st0 = eng.stats()
    launches0, rebuilds0 = int(st0[2]), int(st0[1])
    list_entries, list_tiles = int(st0[5]), int(st0[6])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(os.path.join(args.out_dir, f"clocks_rank{rank}.csv"))
    with clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            ev[k][0].record(stream)
            bench_step()
            ev[k][1].record(stream)
            flush_l2(flush)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if dist is not None:
        dist.barrier()
    st1 = eng.stats()
    launches = int(st1[2]) - launches0
    rebuild_rate = (int(st1[1]) - rebuilds0) / float(run.n_walkers * args.steps * md)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms = float(ms_t.item())
    secs = ms * 1e-3
    value = walker_ns_per_day(run.n_walkers * world, args.steps * md, run.dt, secs)
    pair_rate = pairs_per_md * world * args.steps * md / secs

    # ---- end to end through the C ABI with host buffers ----
    n, W = spec.n, run.n_walkers
    # every walker's state in page-locked buffers, moved with one call each way
    pin_x = torch.empty((W * n, 3), dtype=torch.float32, pin_memory=True)
    pin_v = torch.empty((W * n, 3), dtype=torch.float32, pin_memory=True)
    px, pv = pin_x.numpy(), pin_v.numpy()
    host = eng.get_states(x=px, v=pv)
    lam, plam = host["lam"].copy(), host["plam"].copy()
    h2d = W * (2 * n * 3 * 4 + 16)
    d2h_state = W * (2 * n * 3 * 4 + 16)
    nb = sum(s.n_bins for s in run.stages)
    d2h = d2h_state + nb * (8 + 8 + 8)

    def e2e_step():
        eng.set_states(x=px, v=pv, lam=lam, plam=plam)
        eng.step(md, stream)
        for k in range(len(run.stages)):
            eng.read_abf(0, k)
        st = eng.get_states(x=px, v=pv)
        lam[:], plam[:] = st["lam"], st["plam"]

    e2e_steps = max(2, args.steps)
    e2e_step()
    flush_l2(flush)
    torch.cuda.synchronize()
    te = 0.0
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        te += time.perf_counter() - t0
        flush_l2(flush)
        torch.cuda.synchronize()
    te_t = torch.tensor([te], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(te_t, op=dist.ReduceOp.MAX)
    e2e_val = walker_ns_per_day(run.n_walkers * world, e2e_steps * md, run.dt, float(te_t.item()))

    # ---- plain form (one walker per launch sequence, no graph), same engine ----
    plain_md = max(10, md // 5)
    torch.cuda.synchronize()
    pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eng.step_plain(2, stream)
    pa.record(stream)
    eng.step_plain(plain_md, stream)
    pb.record(stream)
    torch.cuda.synchronize()
    plain_val = walker_ns_per_day(run.n_walkers * world, plain_md, run.dt, pa.elapsed_time(pb) * 1e-3)

    # ---- roofline of the dominant kernel (pair pass), events per kernel ----
    kt = eng.time_kernels(args.profile_steps, stream)
    pair_ms = kt["pairs"][0]
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tflops = n_sm * 128 * 2 * 2.070e9 / 1e12  # FP32 lanes x FMA x max SM clock
    achieved = pairs_per_md * FLOP_PER_PAIR / (pair_ms * 1e-3) / 1e12
    eng.sync()
    csum = clk.summary(local)
    # measured FMA peaks (FP32 and FP64), clocks sampled during them
    peaks = None
    if not args.no_peaks:
        clk2 = ClockSampler(os.path.join(args.out_dir, f"clocks_peaks_rank{rank}.csv"))
        with clk2:
            fp32 = labf.fp_peak(False, 1.0, stream)
            fp64 = labf.fp_peak(True, 0.5, stream)
        peaks = dict(fp32_tflops=fp32, fp64_tflops=fp64, nominal_fp32_tflops=peak_tflops,
                     clocks=clk2.summary(local),
                     note="la_fp_peak: independent FMA chains on every SM, CUDA events, about 1 s (FP32) "
                          "and 0.5 s (FP64) of device time")
    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        extra["C3"] = bench_uneven(args, stream, peak_tflops)
        extra["C5"] = bench_large(args, stream, peak_tflops)
        extra["C4"] = bench_autograd(args)
    # the integrator streams per atom: F (24 B), 1/m and noise scale (8),
    # v (16), x (16), reference x (16), slot indices (8) read; x, v (32) and
    # the cleared F (24) written
    hbm_peak, hbm_src = measured_hbm()
    # 88 B read + 56 B written per atom, plus the 16 B reference position
    # read when pruning is on
    integ_per_atom = 144.0 + (16.0 if args.prune_margin > 0 else 0.0)
    integ_bytes = integ_per_atom * run.n_walkers * spec.n
    integ_gbs = integ_bytes / (kt["integrate"][0] * 1e-3) / 1e9

    m = re.search(r"pair_variant=(\d+)", eng.autotune_report())
    traffic, traffic_src = measured_traffic(int(m.group(1)) if m else -1)
    if rank == 0:
        cb = None
        if world == 1 and not args.no_cpu_baseline:
            cb, _ = cpu_baseline(steps=args.cpu_steps, single_thread=True)
        line = dict(
            metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
            ms_per_step=ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
            dtype="f32", data="synthetic",
            config=dict(workload=workload_name(args.skin, args.prune_margin), walkers=run.n_walkers,
                        atoms_per_walker=spec.n, md_steps_per_bench_step=md, l2="flushed between bench steps (256 MB write)",
                        parallelism="replicas" if world > 1 else "1 GPU, walkers batched",
                        launch=eng.autotune_report(),
                        launch_options=",".join(
                            f"{k}={v}" for k, v in re.findall(r"(pair_variant|pair_ctas_per_sm|chunk_entries)=(\d+)",
                                                              eng.autotune_report()))),
            pair_interactions_per_s=pair_rate,
            in_cutoff_pairs_per_md_step=pairs_per_md,
            lists=dict(rebuilds_per_walker_md_step=rebuild_rate, cluster_pair_entries=list_entries,
                       tiles_8x4=list_tiles, normal_pairs=pairs_n,
                       tile_efficiency=pairs_n / max(1, 32 * list_tiles)),
            plain_form=dict(value=plain_val, unit=UNIT, md_steps=plain_md,
                            note="one walker per launch sequence, no CUDA graph"),
            e2e=dict(value=e2e_val, unit=UNIT, h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                     note="state upload (la_set_states) + la_step_walkers + la_read_abf + la_get_states, "
                          "host<->device copies in the timed region"),
            gpu_launches=launches,
            roofline=dict(bound="alu", achieved=achieved, peak=peak_tflops, unit="TFLOP/s",
                          frac=achieved / peak_tflops, traffic=traffic, traffic_source=traffic_src,
                          kernel="k_pairs, fused step launch (normal + alchemical pairs, bonded, walker, lambda)",
                          pair_kernel_ms=pair_ms,
                          peak_note=f"{n_sm} SMs x 128 FP32 lanes x 2 flop x 2070 MHz (max SM clock), nominal",
                          peak_measured=peaks["fp32_tflops"] if peaks else None,
                          frac_of_measured=achieved / peaks["fp32_tflops"] if peaks else None,
                          flop_per_pair=FLOP_PER_PAIR,
                          kernel_ms=dict((k, v[0]) for k, v in kt.items()),
                          kernel_ms_sum=sum(v[0] for v in kt.values()),
                          md_step_ms=ms / args.steps / md,
                          timing_note="CUDA events on the engine stream between the launches of the batched "
                                      "step as the graph runs them (integrate | gate, and the list kernels on "
                                      "steps where a walker rebuilds | fused pair launch with bonded, walker and "
                                      "lambda work) over --profile-steps steps right after the timed region; "
                                      "kernel_ms_sum against md_step_ms (the graph-timed MD step) leaves the "
                                      "launch gaps"),
            roofline_hbm=dict(bound="hbm", kernel="k_integrate", achieved=integ_gbs, peak=hbm_peak,
                              unit="GB/s", frac=integ_gbs / hbm_peak, bytes_per_launch=integ_bytes,
                              peak_source=hbm_src),
            clocks=csum,
            wall_s=wall,
        )
        if cb is not None:
            line["cpu_baseline"] = cb
        if peaks is not None:
            line["peaks"] = peaks
        line.update(extra)
        print(json.dumps(line))
    eng.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="labf", choices=["labf", "reference"])
    ap.add_argument("--md-steps", type=int, default=200)
    ap.add_argument("--graph-steps", type=int, default=20)
    ap.add_argument("--settle", type=int, default=2000)
    ap.add_argument("--profile-steps", type=int, default=200)
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the uneven-batch, large-complex and differentiation workloads")
    ap.add_argument("--no-peaks", action="store_true", help="skip the FP32/FP64 FMA peak measurement")
    ap.add_argument("--launch", default="",
                    help="fixed pair-kernel shape, e.g. pair_variant=1,pair_ctas_per_sm=6,chunk_entries=64")
    ap.add_argument("--skin", type=float, default=SKIN_NM, help="list skin (nm)")
    ap.add_argument("--prune-margin", type=float, default=PRUNE_NM,
                    help="pair-pass pruning margin (nm); 0 = off")
    ap.add_argument("--out-dir", default=os.path.join(ROOT, "bench_out"), help="clock samples (CSV)")
    args = ap.parse_args()
    os.makedirs(args.out_dir, exist_ok=True)
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
