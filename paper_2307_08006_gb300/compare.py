"""lambda-ABF against fixed-lambda windows at equal cost (Sec. 4), and the
lambda-particle mass / friction sweep (SI S2), on the GPU engine.

Both estimators integrate <dU/dlambda> over lambda (Sec. 2.3): lambda-ABF
from its adaptively biased walkers, the windows method by thermodynamic
integration over walkers frozen at window centres.  At equal cost (the same
number of walkers and MD steps) the spread of Delta A over independent seeds
measures each method's statistical efficiency.

    python -m paper_2307_08006_gb300.compare --system harmonic --seeds 5
    python -m paper_2307_08006_gb300.compare --sweep --steps 200000 --seeds 3
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import replace
from typing import Dict, List, Sequence

import numpy as np

from . import labf, synth


def delta_a_runs(spec, run, lam0, n_steps: int, seeds: Sequence[int], chunk: int = 10000,
                 options=None) -> List[float]:
    """Delta A (sum over stages) after n_steps, one independent run per seed
    (NaN while a bin is still empty)."""
    out = []
    for sd in seeds:
        r = replace(run, seed=int(sd))
        st = synth.initial_state(spec, r, seed=int(sd) + 7, lam0=lam0)
        eng = labf.engine_for(spec, r, st, options=options or dict(graph_steps=20))
        done = 0
        while done < n_steps:
            k = min(chunk, n_steps - done)
            eng.step(k)
            done += k
        out.append(sum(eng.read_abf(0, s)["dA"] for s in range(len(r.stages))))
        eng.close()
    return out


def systems(name: str):
    """(spec, lambda-ABF run, exact Delta A or None) for a named system."""
    if name == "harmonic":
        spec = synth.harmonic_well(dims=1)
        run = synth.harmonic_run(n_walkers=4, n_bins=20)
        return spec, run, 0.5 * np.log(4.0)
    if name == "lj":
        return synth.lj_fluid(), synth.lj_fluid_run(n_walkers=4), None
    if name == "water":
        spec = synth.water_box(256, 4, seed=8010, box=1.984, r_cut=0.85)
        run = synth.water_run(seed=8010, walkers_per_stage=4, n_bins=20)
        return spec, run, None
    raise ValueError(name)


def compare(name: str, n_steps: int, seeds: Sequence[int], windows_per_stage: int) -> Dict:
    spec, run, exact = systems(name)
    per_stage = [s.n_walkers for s in run.stages]
    wpw = max(1, per_stage[0] // windows_per_stage)
    t0 = time.perf_counter()
    abf = delta_a_runs(spec, run, None, n_steps, seeds)
    wrun, lam0 = synth.fixed_lambda_windows(run, windows_per_stage, wpw)
    # equal cost: the same walker-steps in total
    w_steps = int(round(n_steps * run.n_walkers / wrun.n_walkers))
    win = delta_a_runs(spec, wrun, lam0, w_steps, seeds)
    a, w = np.asarray(abf), np.asarray(win)
    res = dict(system=name, seeds=len(seeds), walker_steps=int(n_steps * run.n_walkers),
               labf=dict(mean=float(a.mean()), std=float(a.std(ddof=1)), walkers=run.n_walkers,
                         steps=n_steps),
               windows=dict(mean=float(w.mean()), std=float(w.std(ddof=1)), walkers=wrun.n_walkers,
                            steps=w_steps, windows_per_stage=windows_per_stage),
               variance_ratio_windows_over_labf=float(w.var(ddof=1) / max(a.var(ddof=1), 1e-300)),
               exact=exact, seconds=time.perf_counter() - t0)
    return res


def sweep_system(name: str):
    """(spec, run) of the systems the mass / friction sweep runs on: the
    256-water two-stage system (20 bins per stage) or the 4096-water bench
    workload (100 bins per stage)."""
    if name == "water256":
        spec = synth.water_box(256, 4, seed=8010, box=1.984, r_cut=0.85)
        return spec, synth.water_run(seed=8010, walkers_per_stage=4, n_bins=20)
    if name == "solvation":
        spec = synth.water_box(4096, 12, seed=8007)
        return spec, synth.water_run(seed=8007, walkers_per_stage=8, n_bins=100, n_full=200.0, skin=0.15)
    raise ValueError(name)


def sweep(n_steps: int, seeds: Sequence[int], masses: Sequence[float], frictions: Sequence[float],
          system: str = "water256", every: int = 1000) -> List[Dict]:
    """Delta A (per stage and summed) and lambda mobility for lambda-particle
    masses (kJ/mol ps^2) and frictions (ps^-1), SI S2.  Every (mass,
    friction, seed) is its own system of one batched engine, so the whole
    sweep advances in one launch sequence per step."""
    spec, base = sweep_system(system)
    combos = [(float(m), float(g), int(sd)) for m in masses for g in frictions for sd in seeds]
    inputs = []
    for m, g, sd in combos:
        r = replace(base, m_lambda=m, gamma_lambda=g, seed=sd)
        inputs.append(labf.SystemInput(spec, r, synth.initial_state(spec, r, seed=sd + 7)))
    eng = labf.Engine(inputs, options=dict(graph_steps=20))
    W = eng.n_walkers
    lam_min, lam_max = np.full(W, np.inf), np.full(W, -np.inf)
    done = 0
    while done < n_steps:
        k = min(every, n_steps - done)
        eng.step(k)
        done += k
        lam = eng.get_states()["lam"]
        lam_min, lam_max = np.minimum(lam_min, lam), np.maximum(lam_max, lam)
    per = {}
    w0 = 0
    for si, (m, g, sd) in enumerate(combos):
        nw = inputs[si].run.n_walkers
        abf = [eng.read_abf(si, k) for k in range(len(base.stages))]
        empty = int(sum(int((a["count"] == 0).sum()) for a in abf))
        per.setdefault((m, g), []).append(dict(dA=[a["dA"] for a in abf], empty=empty,
                                               span=float(np.mean(lam_max[w0:w0 + nw] - lam_min[w0:w0 + nw]))))
        w0 += nw
    eng.close()
    rows = []
    for (m, g), rs in per.items():
        ok = [r["dA"] for r in rs if r["empty"] == 0]
        tot = [sum(d) for d in ok]
        rows.append(dict(m_lambda=m, gamma_lambda=g, system=system, steps=n_steps, seeds=len(rs),
                         dA_mean=float(np.mean(tot)) if ok else None,
                         dA_std=float(np.std(tot, ddof=1)) if len(ok) > 1 else None,
                         dA_stage_mean=[float(np.mean([d[k] for d in ok])) for k in range(len(base.stages))]
                         if ok else None,
                         empty_bins=[r["empty"] for r in rs], lambda_span=float(np.mean([r["span"] for r in rs]))))
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--system", default="harmonic", choices=["harmonic", "lj", "water"])
    ap.add_argument("--steps", type=int, default=100000)
    ap.add_argument("--seeds", type=int, default=5)
    ap.add_argument("--windows", type=int, default=10)
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--sweep-system", default="water256", choices=["water256", "solvation"])
    args = ap.parse_args()
    seeds = [8100 + k for k in range(args.seeds)]
    if args.sweep:
        m0 = synth.M_LAMBDA_KJ_PS2
        for row in sweep(args.steps, seeds, [m0 / 10, m0, m0 * 10], [100.0, 1000.0], system=args.sweep_system):
            print(json.dumps(row))
    else:
        print(json.dumps(compare(args.system, args.steps, seeds, args.windows)))


if __name__ == "__main__":
    main()
