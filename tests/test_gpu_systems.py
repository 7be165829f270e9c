"""GPU tests of the workload shapes beyond the single small box: the uneven
batch (8 systems, 64 walkers in one engine), differentiation (autograd
through the engine at 21 lambda values), the large restrained complex
(sampled forces), statistical free-energy parity, and error paths.

Oracle values come from oracle/ only (FP64, O(N^2) or masked O(k N)).
"""
import numpy as np
import pytest

import oracle
from paper_2307_08006_gb300 import labf, synth

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5


def rel_rms(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def jittered(sp, seed, amp=0.01):
    rng = np.random.default_rng(seed)
    sp.x = ((sp.x + rng.normal(0.0, amp, sp.x.shape)) % sp.box).astype(np.float32)
    return sp


def sample_atoms(spec, k, seed, extra=()):
    rng = np.random.default_rng(seed)
    idx = set(rng.choice(spec.n, k, replace=False).tolist()) | set(int(i) for i in extra)
    return np.asarray(sorted(idx))


def check_sampled(eng, walker, spec, x, lam, atoms):
    g = eng.energy_forces(walker)
    ref = oracle.energy_forces_masked(oracle.OracleSystem(spec), x.astype(np.float64), lam, atoms)
    f = g["F"].cpu().numpy().astype(np.float64)[atoms]
    fr = ref["F"][atoms]
    assert rel_rms(f, fr) < FORCE_TOL
    scale = max(1.0, abs(ref["dl"][0]) + abs(ref["dl"][1]) + abs(ref["dl"][2]))
    assert abs(g["dUdl"] - ref["dUdl"]) <= FORCE_TOL * scale
    return g, ref


# ---------------------------------------------------------------------------
# uneven batch: 8 water boxes (256 ... 8192 waters), 8 walkers each
# ---------------------------------------------------------------------------
def _uneven_inputs(n_walkers_per_system=8, seed=8008):
    systems = synth.uneven_batch(seed)
    inputs = []
    for k, sp in enumerate(systems):
        jittered(sp, seed + k)
        run = synth.uneven_run(seed=seed + k, walkers_per_system=n_walkers_per_system)
        lam0 = list(np.linspace(0.05, 0.45, run.stages[0].n_walkers)) + \
            list(np.linspace(0.55, 0.95, run.stages[1].n_walkers))
        inputs.append(labf.SystemInput(sp, run, synth.initial_state(sp, run, lam0=lam0)))
    return inputs


def test_uneven_batch_forces_pairs_and_forms():
    inputs = _uneven_inputs()
    eng = labf.Engine(inputs)
    assert eng.n_walkers == 64
    w = 0
    for k, si in enumerate(inputs):
        atoms = sample_atoms(si.spec, 48, 100 + k, extra=np.nonzero(si.spec.alch)[0])
        for wl in (0, si.run.n_walkers - 1):
            check_sampled(eng, w + wl, si.spec, si.state.x[wl], si.state.lam[wl], atoms)
        w += si.run.n_walkers
    # pair set of the smallest box (r_c = 0.85 nm, several images per cluster pair)
    sp0 = inputs[0].spec
    pairs, kind = eng.get_pairs(0)
    opairs, okind = oracle.pair_set(oracle.OracleSystem(sp0), inputs[0].state.x[0],
                                    sp0.r_cut + inputs[0].run.skin)
    assert np.array_equal(pairs, opairs) and np.array_equal(kind, okind)
    # batched (graph) and plain forms agree bit for bit on the uneven batch
    e2 = labf.Engine(inputs)
    eng.step(25)
    e2.step_plain(25)
    for ww in (0, 9, 31, 63):
        a, b = eng.get_state(ww), e2.get_state(ww)
        assert np.array_equal(a["x"], b["x"]) and a["lam"] == b["lam"]


def test_all_walker_state_calls_match_per_walker_calls():
    """la_get_states / la_set_states over eight systems of different sizes:
    the same values as the per-walker calls, and the same trajectory after
    setting every walker either way (also with x alone)."""
    inputs = _uneven_inputs()
    eng = labf.Engine(inputs)
    eng.step(5)
    st = eng.get_states()
    rows = eng.walker_rows
    assert rows[-1] == sum(si.spec.n * si.run.n_walkers for si in inputs)
    for w in range(eng.n_walkers):
        g = eng.get_state(w)
        r0, r1 = rows[w], rows[w + 1]
        assert np.array_equal(st["x"][r0:r1], g["x"]) and np.array_equal(st["v"][r0:r1], g["v"])
        assert st["lam"][w] == g["lam"] and st["plam"][w] == g["plam"]
    x_new = (st["x"] + np.float32(0.001)).astype(np.float32)
    v_new = (st["v"] * np.float32(0.5)).astype(np.float32)
    plam_new = -st["plam"]
    e1, e2 = labf.Engine(inputs), labf.Engine(inputs)
    e1.set_states(x=x_new, v=v_new, lam=st["lam"], plam=plam_new)
    for w in range(e2.n_walkers):
        r0, r1 = rows[w], rows[w + 1]
        e2.set_state(w, x=x_new[r0:r1], v=v_new[r0:r1], lam=st["lam"][w], plam=plam_new[w])
    e1.step(7)
    e2.step(7)
    a, b = e1.get_states(), e2.get_states()
    for k in ("x", "v", "lam", "plam"):
        assert np.array_equal(a[k], b[k]), k
    # positions alone: velocities stay
    e1.set_states(x=b["x"])
    c = e1.get_states()
    assert np.array_equal(c["x"], b["x"]) and np.array_equal(c["v"], a["v"])


def test_uneven_batch_pruning_bit_identical():
    """Pruning in the batched pair pass on eight systems of different sizes
    and cutoffs (each with its own margin threshold and re-pruning trigger):
    the same bits as the unpruned one-walker-per-launch form."""
    inputs = _uneven_inputs()
    a = labf.Engine(inputs, options=dict(prune_margin=0.05))
    b = labf.Engine(inputs)
    a.step(40)
    b.step_plain(40)
    for ww in (0, 9, 17, 31, 40, 63):
        ga, gb = a.get_state(ww), b.get_state(ww)
        assert np.array_equal(ga["x"], gb["x"]) and np.array_equal(ga["v"], gb["v"])
        assert ga["lam"] == gb["lam"] and ga["plam"] == gb["plam"]
    assert int(a.stats()[6]) < int(b.stats()[6])


# ---------------------------------------------------------------------------
# differentiation: U(x, lambda, theta) through torch.autograd at 21 lambdas
# ---------------------------------------------------------------------------
def test_autograd_gradients_match_oracle_at_21_lambdas():
    import torch

    from paper_2307_08006_gb300 import autograd

    sp = jittered(synth.water_box(4096, 12, seed=8009), 8009)
    run = synth.water_run(seed=8009, walkers_per_stage=1)
    run.stages = [synth.Stage(0.0, 1.0, 20, 1)]
    state = synth.initial_state(sp, run, lam0=[0.0])
    eng = labf.engine_for(sp, run, state)
    dev = torch.device("cuda", 0)
    osys = oracle.OracleSystem(sp)
    atoms = sample_atoms(sp, 64, 7, extra=np.nonzero(sp.alch)[0])
    theta0 = autograd.theta_of(sp)
    n_alch = theta0.shape[0]
    for lam in np.linspace(0.0, 1.0, 21):
        x = torch.tensor(state.x[0], device=dev, requires_grad=True)
        lt = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
        th = torch.tensor(theta0, dtype=torch.float64, device=dev, requires_grad=True)
        U = autograd.energy(eng, 0, x, lt, th)
        gx, gl, gth = torch.autograd.grad(U, [x, lt, th])
        ref = oracle.energy_forces_masked(osys, state.x[0].astype(np.float64), lam, atoms)
        fx = -gx.cpu().numpy().astype(np.float64)[atoms]
        assert rel_rms(fx, ref["F"][atoms]) < FORCE_TOL
        dscale = max(1.0, abs(ref["dl"][0]) + abs(ref["dl"][1]) + abs(ref["dl"][2]))
        assert abs(float(gl) - ref["dUdl"]) <= FORCE_TOL * dscale
        rth = ref["dth"][:3 * n_alch].reshape(n_alch, 3)
        tscale = max(1.0, float(np.abs(rth).max()))
        np.testing.assert_allclose(gth.cpu().numpy(), rth, rtol=1e-4, atol=1e-5 * tscale)
        # second derivatives d2U/dlambda dtheta from the same pass
        g = eng.energy_forces(0)
        r2 = ref["d2th"][:3 * n_alch]
        np.testing.assert_allclose(g["d2th"][:3 * n_alch], r2, rtol=1e-4,
                                   atol=1e-5 * max(1.0, float(np.abs(r2).max())))


# ---------------------------------------------------------------------------
# the benchmark's own workload and launch configuration, full size
# ---------------------------------------------------------------------------
def test_bench_workload_full_size():
    """16 walkers x 12 300 atoms with the bench's options (autotuned pair
    kernel, 20-step CUDA graph with the fused pair launch): 20 graph steps
    are bit-identical to 20 steps of the one-walker-per-launch form, and
    sampled forces and dU/dlambda of three walkers match the oracle."""
    import bench

    spec, run = bench.workload()
    state = synth.initial_state(spec, run)
    e1 = labf.Engine([labf.SystemInput(spec, run, state)], options=dict(graph_steps=20, autotune=1))
    e2 = labf.Engine([labf.SystemInput(spec, run, state)], options=dict(graph_steps=20))
    e1.step(20)
    e2.step_plain(20)
    assert e1.sync() == 0 and e2.sync() == 0
    for w in range(run.n_walkers):
        a, b = e1.get_state(w), e2.get_state(w)
        assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["v"], b["v"])
        assert a["lam"] == b["lam"] and a["plam"] == b["plam"]
    atoms = sample_atoms(spec, 48, 13, extra=np.nonzero(spec.alch)[0])
    for w in (0, 9, 15):
        s = e1.get_state(w)
        check_sampled(e1, w, spec, s["x"], s["lam"], atoms)


# ---------------------------------------------------------------------------
# large restrained complex: 96k atoms, sampled forces (incl. restraints)
# ---------------------------------------------------------------------------
def test_large_complex_sampled_forces_and_steps():
    sp = synth.large_complex()
    run = synth.large_complex_run(walkers_per_stage=1)
    state = synth.initial_state(sp, run, lam0=[0.3, 0.7])
    eng = labf.engine_for(sp, run, state)
    lig = np.nonzero(sp.alch)[0]
    atoms = sample_atoms(sp, 40, 11, extra=list(lig[:8]) + list(sp.fb_b[:8]) + list(sp.posres_idx[:8]))
    for w in range(2):
        check_sampled(eng, w, sp, state.x[w], state.lam[w], atoms)
    eng.step(40)
    eng.sync()
    s = eng.get_state(1)
    check_sampled(eng, 1, sp, s["x"], s["lam"], atoms)


# ---------------------------------------------------------------------------
# free energy: closed form on the GPU, and GPU vs oracle statistics
# ---------------------------------------------------------------------------
@pytest.mark.slow
def test_harmonic_switch_free_energy_and_theta_gradient_on_gpu():
    """Delta A = (kT/2) ln(k1/k0) within 0.05 kT and d Delta A / d k1 =
    kT / (2 k1) from the GPU accumulator (1-D well, 4 walkers, 3 seeds)."""
    vals, grads = [], []
    for seed in range(3):
        sp = synth.harmonic_well(dims=1, k0=1.0, k1=4.0)
        run = synth.harmonic_run(seed=300 + seed, n_walkers=4)
        run.theta_stats = True
        eng = labf.engine_for(sp, run)
        eng.step(250_000)
        a = eng.read_abf(0, 0)
        assert not a["empty_bin"]
        vals.append(a["dA"])
        grads.append(eng.read_theta(0, 0)["dA_dtheta"][-1])
    assert np.mean(vals) == pytest.approx(0.5 * np.log(4.0), abs=0.05)
    assert np.mean(grads) == pytest.approx(1.0 / 8.0, abs=0.02)


@pytest.mark.slow
def test_lj_fluid_delta_a_gpu_vs_oracle_two_combined_se():
    """Delta A of the LJ-fluid workload from GPU and oracle runs (8 seeds
    each, 20 000 steps, 4 walkers) agree within two combined standard errors."""
    oracle.set_threads(4)
    res = {"gpu": [], "cpu": []}
    for seed in range(8):
        sp = synth.lj_fluid()
        run = synth.lj_fluid_run(seed=500 + seed)
        st = synth.initial_state(sp, run)
        eng = labf.engine_for(sp, run, st)
        eng.step(20_000)
        a = eng.read_abf(0, 0)
        assert not a["empty_bin"]
        res["gpu"].append(a["dA"])
        sim = oracle.Simulation(sp, run, st)
        sim.run(20_000)
        res["cpu"].append(sim.delta_a(0)[2])
    g, c = np.asarray(res["gpu"]), np.asarray(res["cpu"])
    se = np.sqrt(g.var(ddof=1) / len(g) + c.var(ddof=1) / len(c))
    assert abs(g.mean() - c.mean()) <= 2.0 * se + 1e-9, (g.mean(), c.mean(), se)


def test_shared_freq_merge_matches_oracle():
    sp = jittered(synth.water_box(100, 6, seed=61, box=1.5, r_cut=0.6), 61)
    run = synth.water_run(seed=62, walkers_per_stage=2, n_bins=10)
    run.shared_freq = 4
    st = synth.initial_state(sp, run, lam0=[0.1, 0.3, 0.6, 0.8])
    eng = labf.engine_for(sp, run, st)
    sim = oracle.Simulation(sp, run, st)
    for n in (3, 5):
        eng.step(n)
        sim.run(n)
        for stage in range(2):
            a = eng.read_abf(0, stage)
            s, _, c = sim.stage_bins(stage)
            assert np.array_equal(a["count"], c)
            np.testing.assert_allclose(a["sum"], s, rtol=1e-4, atol=1e-3 * max(1.0, np.abs(s).max()))


# ---------------------------------------------------------------------------
# fixed-lambda windows (Sec. 4 comparison method) and the equal-cost comparison
# ---------------------------------------------------------------------------
def test_fixed_lambda_windows_closed_form():
    sp = synth.harmonic_well(dims=3)
    run, lam0 = synth.fixed_lambda_windows(synth.harmonic_run(seed=311), 10, 4)
    st = synth.initial_state(sp, run, lam0=lam0)
    eng = labf.engine_for(sp, run, st, options=dict(graph_steps=20))
    eng.step(100_000)
    assert [eng.get_state(w)["lam"] for w in range(run.n_walkers)] == lam0  # frozen
    r = eng.read_abf(0, 0)
    lc = (np.arange(10) + 0.5) / 10
    np.testing.assert_allclose(r["grad"], 1.5 * 3.0 / (1.0 + 3.0 * lc), rtol=0.08)
    assert abs(r["dA"] - 1.5 * np.log(4.0)) < 0.05


def test_labf_and_windows_at_equal_cost():
    from paper_2307_08006_gb300 import compare
    res = compare.compare("harmonic", 200_000, [8100, 8101, 8102], 4)
    exact = 0.5 * np.log(4.0)
    assert res["labf"]["walkers"] == res["windows"]["walkers"] == 4
    assert res["labf"]["steps"] == res["windows"]["steps"]
    assert abs(res["labf"]["mean"] - exact) < 0.05
    assert abs(res["windows"]["mean"] - exact) < 0.05
    assert res["variance_ratio_windows_over_labf"] > 0


# ---------------------------------------------------------------------------
# host-level sharing across engines (Sec. 2.4 walkers on several GPUs)
# ---------------------------------------------------------------------------
def _sharing_inputs(seed, shared_freq):
    sp = jittered(synth.water_box(100, 6, seed=91, box=1.5, r_cut=0.6), 91)
    run = synth.water_run(seed=seed, walkers_per_stage=2, n_bins=10)
    run.shared_freq = shared_freq
    st = synth.initial_state(sp, run, lam0=[0.1, 0.3, 0.6, 0.8])
    return sp, run, st


def test_export_import_equals_device_merge():
    K = 6
    sp, run_h, st = _sharing_inputs(92, 0)
    _, run_d, _ = _sharing_inputs(92, K)
    host = labf.engine_for(sp, run_h, st, options=dict(autotune=0))
    dev = labf.engine_for(sp, run_d, st, options=dict(autotune=0))
    # identical until the device merge at step K (the samples of step K are
    # folded before it), so the host's export must equal the merged result
    host.step(K)
    dev.step(K)
    for stage in range(2):
        assert host.read_abf(0, stage)["count"].sum() == 0
        s1, s2, c = host.abf_export(0, stage)
        d = dev.read_abf(0, stage)
        assert c.sum() == K * 2
        assert np.array_equal(c, d["count"])
        assert np.array_equal(s1, d["sum"]) and np.array_equal(s2, d["sumsq"])
        host.abf_import(s1, s2, c, 0, stage)
        h = host.read_abf(0, stage)
        for key in ("sum", "sumsq", "count", "grad"):
            assert np.array_equal(np.nan_to_num(h[key]), np.nan_to_num(d[key]))
        z = host.abf_export(0, stage)
        assert not any(np.any(a) for a in z)
    with pytest.raises(labf.LabfError):
        host.abf_import(s1, s2, -np.ones_like(c), 0, 0)
    buf = np.zeros(16)
    cnt = np.zeros(16, np.int64)
    rc = host.lib.la_abf_export(host.handle, 0, 5, labf._p(buf), labf._p(buf), labf._p(cnt), None)
    assert rc == -1  # LA_ERR_INVALID_ARG: no stage 5


def test_two_engines_share_statistics_in_rank_order():
    from paper_2307_08006_gb300 import multiwalker
    engines = []
    for seed in (93, 94):
        sp, run, st = _sharing_inputs(seed, 0)
        engines.append(labf.engine_for(sp, run, st))
    rounds, every = 3, 5
    for _ in range(rounds):
        for e in engines:
            e.step(every)
        for stage in range(2):
            parts = [e.abf_export(0, stage) for e in engines]
            tot = [multiwalker.reduce_in_rank_order([p[j] for p in parts]) for j in range(3)]
            for e in engines:
                e.abf_import(*tot, sys=0, stage=stage)
    for stage in range(2):
        a, b = engines[0].read_abf(0, stage), engines[1].read_abf(0, stage)
        for key in ("sum", "sumsq", "count"):
            assert np.array_equal(a[key], b[key])
        assert int(a["count"].sum()) == rounds * every * 2 * len(engines)
    # distinct seeds: the walkers do not move alike
    assert not np.array_equal(engines[0].get_state(0)["x"], engines[1].get_state(0)["x"])


# ---------------------------------------------------------------------------
# error paths (no GPU fault: every write is bounds-checked, the status word
# reports the condition)
# ---------------------------------------------------------------------------
def test_list_overflow_is_reported():
    sp = jittered(synth.water_box(100, 6, seed=71, box=1.5, r_cut=0.6), 71)
    # all atoms squeezed into a corner: capacities are sized for the box's
    # average density, so the alchemical lists overflow at the first build
    sp.x = (sp.x * 0.4).astype(np.float32)
    run = synth.water_run(seed=72, walkers_per_stage=1, n_bins=10)
    with pytest.raises(labf.LabfError) as ei:
        labf.engine_for(sp, run, options=dict(list_capacity_factor=1.0))
    assert ei.value.code in (-6, -7, -8)


def test_nonfinite_state_is_reported():
    sp = jittered(synth.water_box(100, 6, seed=81, box=1.5, r_cut=0.6), 81)
    run = synth.water_run(seed=82, walkers_per_stage=1, n_bins=10)
    eng = labf.engine_for(sp, run)
    s = eng.get_state(0)
    x = s["x"].copy()
    x[5, 1] = np.nan
    eng.set_state(0, x=x)
    with pytest.raises(labf.LabfError) as ei:
        eng.step(2)
        eng.sync()
    assert ei.value.code in (-7, -8, -9)
    with pytest.raises(labf.LabfError):
        eng.step(1)  # sticky
