"""GPU parity: the CUDA engine (through the C ABI) against the FP64 oracle on
identical seeded inputs.

Bars: pair sets bit-exact (integer definition); forces within 1e-5 relative
RMS; dU/dlambda and energy terms within 1e-5 relative to their scale;
lambda path exact; short trajectories (same Philox streams) within FP32
rounding growth; batched and one-walker-per-launch forms bit-identical;
repeated runs bit-identical.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_2307_08006_gb300 import labf, synth

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5


def rel_rms(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def small_water(n_w=100, n_s=6, box=1.5, rc=0.6, seed=31, jitter=0.0):
    sp = synth.water_box(n_w, n_s, seed=seed, box=box, r_cut=rc)
    if jitter:
        rng = np.random.default_rng(seed)
        sp.x = ((sp.x + rng.normal(0, jitter, sp.x.shape)) % box).astype(np.float32)
    return sp


def make_engine(spec, run, lam0=None, state=None, **opt):
    st = state if state is not None else synth.initial_state(spec, run, lam0=lam0)
    return labf.engine_for(spec, run, st, options=opt or None), st


def check_forces(eng, spec, st, walker, lam=None, tol=FORCE_TOL):
    osys = oracle.OracleSystem(spec)
    g = eng.energy_forces(walker)
    ref = oracle.energy_forces(osys, st.x[walker].astype(np.float64), st.lam[walker] if lam is None else lam)
    f = g["F"].cpu().numpy().astype(np.float64)
    assert rel_rms(f, ref["F"]) < tol
    scale = max(1.0, float(np.abs(ref["terms"]).max()))
    np.testing.assert_allclose(g["terms"], ref["terms"], rtol=tol, atol=tol * scale)
    dscale = max(1.0, abs(ref["dl"][0]) + abs(ref["dl"][1]) + abs(ref["dl"][2]))
    assert abs(g["dUdl"] - ref["dUdl"]) <= tol * dscale
    return g, ref


# ---------------------------------------------------------------------------
def test_lambda_path_device_matches_table_and_oracle():
    sp = small_water()
    eng, _ = make_engine(sp, synth.water_run(walkers_per_stage=1))
    rows = read_golden("lambda_schedule_tableS1.txt")
    lam = np.array([float(r[0]) for r in rows])
    out = eng.lambda_path(lam, 0.5, 0.5)
    np.testing.assert_allclose(out[:, 0], [float(r[2]) for r in rows], atol=1e-12)
    np.testing.assert_allclose(out[:, 1], [float(r[1]) for r in rows], atol=1e-12)
    rng = np.random.default_rng(1)
    for bv, be in ((0.5, 0.5), (1.0, 0.0), (0.7, 0.3)):
        lam = np.concatenate([rng.uniform(0, 1, 500), [0.0, 1.0, bv, be]])
        out = eng.lambda_path(lam, bv, be)
        ref = np.array([oracle.lambda_path(v, bv, be) for v in lam])
        assert np.array_equal(out, ref)


@pytest.mark.parametrize("case", ["water_small", "water_ragged", "water_min_box", "lj_fluid"])
def test_pair_set_bit_exact(case):
    if case == "water_small":
        sp, run = small_water(jitter=0.02), synth.water_run(walkers_per_stage=1)
    elif case == "water_ragged":
        sp, run = small_water(n_w=137, n_s=5, box=1.7, seed=5, jitter=0.03), synth.water_run(walkers_per_stage=1)
    elif case == "water_min_box":
        # box just above 2 r_list: several periodic images per cluster pair
        sp = small_water(n_w=64, n_s=4, box=1.25, rc=0.52, seed=7, jitter=0.02)
        run = synth.water_run(walkers_per_stage=1, skin=0.1)
    else:
        sp, run = synth.lj_fluid(), synth.lj_fluid_run(n_walkers=2)
    eng, st = make_engine(sp, run)
    osys = oracle.OracleSystem(sp)
    for w in range(run.n_walkers):
        pairs, kind = eng.get_pairs(w)
        opairs, okind = oracle.pair_set(osys, st.x[w], sp.r_cut + run.skin)
        assert len(pairs) == len(opairs)
        assert np.array_equal(pairs, opairs)
        assert np.array_equal(kind, okind)


def tie_system():
    """Atom pairs placed on the quantization grid of a 1 nm box at D == R
    (not listed), D == R - 1 (listed) and D == R + 1, along the axes and on
    diagonals (600-800-1000 and 480-600-640-1000 triples), some across the
    periodic boundary; R = 10^12 (r_list = 10^6 grid units)."""
    d = 1_000_000
    offs = [(d, 0, 0), (d - 1, 0, 0), (d + 1, 0, 0), (0, -d, 0), (0, -(d - 1), 0), (0, 0, d),
            (0, 0, -(d - 1)), (600000, 800000, 0), (600000, 799999, 0), (600000, 800001, 0),
            (-800000, 0, 600000), (-799999, 0, 600000), (480000, 600000, 640000),
            (480000, 600000, 639999), (-480000, -600000, 640001), (480000, -599999, -640000)]
    g, U = 4194304, 2 ** 24  # groups a quarter box apart; bases near the upper edge wrap
    u = []
    for k in range(64):
        b = np.array([(k % 4) * g + U - 300000, ((k // 4) % 4) * g + U - 300000, (k // 16) * g + 150000])
        u.append(b % U)
        u.append((b + np.array(offs[k % 16])) % U)
    u = np.array(u, np.int64)
    n = len(u)
    x = (u * 2.0 ** -24).astype(np.float32)  # exact: 24 significant bits at most
    sp = synth.SystemSpec(name="ties", box=1.0, mass=np.ones(n), charge=np.zeros(n),
                          sigma=np.full(n, 0.001), epsilon=np.zeros(n), alch=np.zeros(n, np.uint8),
                          excl_group=np.full(n, -1, np.int32), excl_extra=np.full((n, 4), -1, np.int32),
                          x=x, r_cut=800000 * 2.0 ** -24)
    run = dataclasses.replace(synth.lj_fluid_run(n_walkers=1), skin=200000 * 2.0 ** -24)
    expect = sum(1 for k in range(64) if sum(c * c for c in offs[k % 16]) < d * d)
    return sp, run, expect


def test_pair_set_exact_ties():
    sp, run, expect = tie_system()
    osys = oracle.OracleSystem(sp)
    opairs, okind = oracle.pair_set(osys, sp.x, sp.r_cut + run.skin)
    assert len(opairs) == expect == 28
    eng, st = make_engine(sp, run)
    pairs, kind = eng.get_pairs(0)
    assert np.array_equal(pairs, opairs)
    assert np.array_equal(kind, okind)


@pytest.mark.parametrize("lam0", [[0.0, 0.13, 0.37, 0.5], [0.5, 0.62, 0.91, 1.0]])
def test_forces_energies_dudl_water(lam0):
    sp = small_water(jitter=0.01)
    run = synth.water_run(walkers_per_stage=2, n_bins=20)
    eng, st = make_engine(sp, run, lam0=lam0)
    for w in range(run.n_walkers):
        check_forces(eng, sp, st, w)


@pytest.mark.parametrize("n,m", [(2, 1), (1, 2), (2, 2)])
def test_softcore_powers(n, m):
    """Soft-core exponents other than the default (Sec. 3.1.2): forces, energy
    terms, dU/dlambda and the theta derivatives against the oracle."""
    sp = synth.with_changes(small_water(jitter=0.01), sc_n=n, sc_m=m)
    run = synth.water_run(walkers_per_stage=2, n_bins=20)
    eng, st = make_engine(sp, run, lam0=[0.02, 0.21, 0.44, 0.5])
    osys = oracle.OracleSystem(sp)
    for w in range(run.n_walkers):
        g, ref = check_forces(eng, sp, st, w)
        for key in ("dth", "d2th"):
            scale = max(1.0, float(np.abs(ref[key]).max()))
            np.testing.assert_allclose(g[key], ref[key], rtol=1e-4, atol=1e-5 * scale)


def test_forces_lj_fluid():
    sp = synth.lj_fluid()
    run = synth.lj_fluid_run(n_walkers=4)
    eng, st = make_engine(sp, run, lam0=[0.0, 0.3, 0.75, 1.0])
    for w in range(4):
        check_forces(eng, sp, st, w)


@pytest.mark.parametrize("lam0", [[0.03, 0.25, 0.45, 0.5], [0.5, 0.55, 0.74, 0.98]])
def test_restraint_terms(lam0):
    """Positional, flat-bottom COM, lambda-switched well and lambda-dependent
    distance restraints (Sec. 3.1 restraint set) against the oracle."""
    sp = small_water(jitter=0.01)
    n = sp.n
    x = sp.x.astype(np.float64)
    sp = synth.with_changes(
        sp, posres_idx=np.array([0, 3], np.int32), posres_x0=x[[0, 3]] + 0.05, posres_k=1000.0,
        fb_a=np.arange(n - 4, n, dtype=np.int32), fb_b=np.array([6, 9, 12], np.int32),
        fb_d0=0.05, fb_k=800.0, lh_idx=np.array([n - 1], np.int32), lh_x0=x[[n - 1]] + 0.07,
        lh_k0=100.0, lh_k1=400.0, lh_dims=3, lr_ij=np.array([[n - 3, 9], [2, 20], [n - 1, 40]], np.int32),
        lr_delta=1.2, lr_k=500.0)
    run = synth.water_run(walkers_per_stage=2, n_bins=20)
    eng, st = make_engine(sp, run, lam0=lam0)
    no_lr = oracle.OracleSystem(synth.with_changes(sp, lr_ij=np.zeros((0, 2), np.int32)))
    active = 0
    for w in range(run.n_walkers):
        g, ref = check_forces(eng, sp, st, w)
        r0 = oracle.energy_forces(no_lr, st.x[w].astype(np.float64), st.lam[w])
        active += ref["terms"][6] != r0["terms"][6]
    assert active > 0  # the distance restraints act at some of these lambdas


def test_theta_derivatives():
    sp = small_water(jitter=0.01)
    run = synth.water_run(walkers_per_stage=2, n_bins=20)
    eng, st = make_engine(sp, run, lam0=[0.15, 0.4, 0.6, 0.85])
    osys = oracle.OracleSystem(sp)
    for w in range(4):
        g = eng.energy_forces(w)
        ref = oracle.energy_forces(osys, st.x[w].astype(np.float64), st.lam[w])
        for key in ("dth", "d2th"):
            scale = max(1.0, float(np.abs(ref[key]).max()))
            np.testing.assert_allclose(g[key], ref[key], rtol=1e-4, atol=1e-5 * scale)


def test_short_trajectory_matches_oracle():
    sp = small_water(jitter=0.01)
    run = synth.water_run(walkers_per_stage=2, n_bins=20)
    st = synth.initial_state(sp, run, lam0=[0.1, 0.3, 0.6, 0.8])
    eng, _ = make_engine(sp, run, state=st)
    sim = oracle.Simulation(sp, run, st)
    for chunk in (1, 2, 3):
        eng.step(chunk)
        sim.run(chunk)
        for w in range(run.n_walkers):
            s = eng.get_state(w)
            d = s["x"] - sim.a["x"][w]
            d -= sp.box * np.round(d / sp.box)
            assert np.abs(d).max() < 2e-5
            assert np.abs(s["v"] - sim.a["v"][w]).max() < 2e-3 * np.abs(sim.a["v"][w]).max()
            assert s["lam"] == pytest.approx(sim.a["lam"][w], abs=1e-7)
    for stage in range(2):
        a = eng.read_abf(0, stage)
        s, _, c = sim.stage_bins(stage)
        assert np.array_equal(a["count"], c)
        np.testing.assert_allclose(a["sum"], s, rtol=1e-4, atol=1e-3 * np.abs(s).max())


def test_batched_and_plain_forms_are_bit_identical():
    sp = small_water(jitter=0.01)
    run = synth.water_run(walkers_per_stage=2, n_bins=20)
    st = synth.initial_state(sp, run, lam0=[0.1, 0.3, 0.6, 0.8])
    e1, _ = make_engine(sp, run, state=st, graph_steps=4)
    e2, _ = make_engine(sp, run, state=st, graph_steps=4)
    e3, _ = make_engine(sp, run, state=st, graph_steps=-1)  # batched launches, no graph
    e1.step(23)
    e2.step_plain(23)
    e3.step(23)
    for w in range(run.n_walkers):
        a, b, c = e1.get_state(w), e2.get_state(w), e3.get_state(w)
        assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["v"], b["v"])
        assert np.array_equal(a["x"], c["x"]) and np.array_equal(a["v"], c["v"])
        assert a["lam"] == b["lam"] == c["lam"] and a["plam"] == b["plam"] == c["plam"]
        assert a["step"] == b["step"] == c["step"] == 23
    for stage in range(2):
        ra, rb = e1.read_abf(0, stage), e2.read_abf(0, stage)
        assert np.array_equal(ra["sum"], rb["sum"]) and np.array_equal(ra["count"], rb["count"])


def test_repeat_runs_bit_identical():
    sp = small_water(jitter=0.01)
    run = synth.water_run(walkers_per_stage=2, n_bins=20)
    st = synth.initial_state(sp, run, lam0=[0.1, 0.3, 0.6, 0.8])
    outs = []
    for _ in range(2):
        e, _ = make_engine(sp, run, state=st)
        e.step(40)
        outs.append([e.get_state(w) for w in range(4)] + [e.energy_forces(0)["F"].cpu().numpy()])
    for a, b in zip(outs[0][:4], outs[1][:4]):
        assert np.array_equal(a["x"], b["x"]) and a["lam"] == b["lam"]
    assert np.array_equal(outs[0][4], outs[1][4])


def test_pair_kernel_launch_shapes_bit_identical():
    """Every pair-kernel variant, grid size and work-item size gives the same
    bits (per-tile arithmetic is shared; 64-bit fixed-point sums are
    order-free)."""
    sp = small_water(n_w=137, n_s=5, box=1.7, seed=5, jitter=0.03)
    run = synth.water_run(walkers_per_stage=2, n_bins=20)
    st = synth.initial_state(sp, run, lam0=[0.1, 0.3, 0.6, 0.8])
    outs = []
    shapes = [(0, 4, 32), (1, 7, 32), (2, 8, 64), (1, 2, 64), (0, 1, 32), (2, 3, 96), (1, 6, 64)]
    assert {v for v, _, _ in shapes} == set(range(labf.LA_PAIR_VARIANTS))
    for var, ctas, chunk in shapes:
        e, _ = make_engine(sp, run, state=st, pair_variant=var, pair_ctas_per_sm=ctas, chunk_entries=chunk)
        e.step(30)
        outs.append([e.get_state(w) for w in range(4)])
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["v"], b["v"])
            assert a["lam"] == b["lam"] and a["plam"] == b["plam"]
    with pytest.raises(labf.LabfError):
        make_engine(sp, run, state=st, pair_variant=labf.LA_PAIR_VARIANTS)
    with pytest.raises(labf.LabfError):
        make_engine(sp, run, state=st, chunk_entries=48)


@pytest.mark.parametrize("variant", range(labf.LA_PAIR_VARIANTS))
def test_dynamic_pruning_skips_tiles_without_changing_results(variant):
    """The batched step's pair pass re-prunes a walker's tiles (keeping those
    with a listed pair within r_c + margin) whenever one of its atoms moved
    0.45 margin, and skips the pruned tiles until then: fewer tiles, the same
    bits as without pruning and as the one-walker-per-launch form, for every
    kernel variant."""
    sp = small_water(n_w=137, n_s=5, box=1.7, seed=5, jitter=0.03)
    run = synth.water_run(walkers_per_stage=2, n_bins=20, skin=0.15)
    st = synth.initial_state(sp, run, lam0=[0.1, 0.3, 0.6, 0.8])
    eng = {m: make_engine(sp, run, state=st, graph_steps=8, prune_margin=m, pair_variant=variant)[0]
           for m in (0.0, 0.05, 0.1)}
    plain, _ = make_engine(sp, run, state=st, graph_steps=8)
    for e in eng.values():
        e.step(57)
    plain.step_plain(57)
    tiles = {m: int(e.stats()[6]) for m, e in eng.items()}
    assert tiles[0.05] < tiles[0.0] and tiles[0.1] <= tiles[0.0]
    for w in range(run.n_walkers):
        ref = plain.get_state(w)
        for e in eng.values():
            a = e.get_state(w)
            assert np.array_equal(a["x"], ref["x"]) and np.array_equal(a["v"], ref["v"])
            assert a["lam"] == ref["lam"] and a["plam"] == ref["plam"]


def test_dynamic_pruning_across_forms_and_state_changes():
    """Pruned masks stay valid when the batched step alternates with the
    one-walker-per-launch form, the no-graph form and the kernel timer, and
    when a walker's state is replaced: bit-identical to an engine without
    pruning driven the same way."""
    sp = small_water(n_w=137, n_s=5, box=1.7, seed=9, jitter=0.03)
    run = synth.water_run(walkers_per_stage=2, n_bins=20, skin=0.15)
    st = synth.initial_state(sp, run, lam0=[0.05, 0.35, 0.55, 0.9])
    a, _ = make_engine(sp, run, state=st, graph_steps=6, prune_margin=0.04)
    b, _ = make_engine(sp, run, state=st, graph_steps=6)
    c, _ = make_engine(sp, run, state=st, graph_steps=-1, prune_margin=0.04)
    for e in (a, b, c):
        e.step(23)
        e.step_plain(5)
        e.step(17)
        e.time_kernels(4)
        e.step(9)
    s2 = b.get_state(2)
    for e in (a, b, c):
        e.set_state(2, x=s2["x"] + np.float32(0.002), v=s2["v"])
        e.step(31)
    for w in range(run.n_walkers):
        ref = b.get_state(w)
        for e in (a, c):
            g = e.get_state(w)
            assert np.array_equal(g["x"], ref["x"]) and np.array_equal(g["v"], ref["v"])
            assert g["lam"] == ref["lam"] and g["plam"] == ref["plam"]
    assert int(a.stats()[6]) < int(b.stats()[6])


def test_autotune_leaves_the_trajectory_unchanged():
    sp = small_water(jitter=0.01)
    run = synth.water_run(walkers_per_stage=2, n_bins=20)
    st = synth.initial_state(sp, run, lam0=[0.1, 0.3, 0.6, 0.8])
    e1, _ = make_engine(sp, run, state=st, graph_steps=4)
    e2, _ = make_engine(sp, run, state=st, graph_steps=4, autotune=1)
    e1.step(13)
    e2.step(13)
    rep = e2.autotune()
    assert rep.startswith("autotuned")
    e1.step(11)
    e2.step(11)
    for w in range(run.n_walkers):
        a, b = e1.get_state(w), e2.get_state(w)
        assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["v"], b["v"])
        assert a["lam"] == b["lam"] and a["plam"] == b["plam"]
    for stage in range(2):
        ra, rb = e1.read_abf(0, stage), e2.read_abf(0, stage)
        assert np.array_equal(ra["sum"], rb["sum"]) and np.array_equal(ra["count"], rb["count"])


def test_maximum_walkers_and_boundary_lambdas():
    """256 walkers (the per-handle maximum) in one batched launch, lambda
    starting exactly on the stage walls, and the empty-bin warning before
    any sample."""
    sp = synth.lj_fluid()
    run = synth.lj_fluid_run(n_walkers=labf.LA_MAX_WALKERS)
    lam0 = list(np.linspace(0.0, 1.0, run.n_walkers))
    eng, st = make_engine(sp, run, lam0=lam0)
    r = eng.read_abf(0, 0)
    assert r["empty_bin"] and np.isnan(r["grad"]).all() and r["count"].sum() == 0
    for w in (0, 137, run.n_walkers - 1):
        check_forces(eng, sp, st, w)
    eng.step(25)
    assert eng.sync() == 0
    assert int(eng.read_abf(0, 0)["count"].sum()) == 25 * run.n_walkers
    lams = np.array([eng.get_state(w)["lam"] for w in range(run.n_walkers)])
    assert np.all((lams >= 0.0) & (lams <= 1.0))


def test_single_atom_system_and_rebuilds():
    sp = synth.harmonic_well(dims=3)
    run = synth.harmonic_run(n_walkers=4)
    eng, st = make_engine(sp, run)
    eng.step(200)
    eng.sync()
    sim = oracle.Simulation(sp, run, st)
    sim.run(200)
    for w in range(4):
        s = eng.get_state(w)
        assert np.abs(s["x"] - sim.a["x"][w]).max() < 1e-3
        assert s["lam"] == pytest.approx(sim.a["lam"][w], abs=1e-4)


def test_system_without_alchemical_atoms():
    """Degenerate case: no alchemical atom (pure water).  dU/dlambda is 0 for
    every walker, every force and energy term and the pair set still match the
    oracle, the ABF bins collect exact zeros, and the batched and plain forms
    agree bit for bit."""
    sp = small_water(n_w=120, n_s=0, box=1.6, seed=9, jitter=0.02)
    assert int(sp.alch.sum()) == 0
    run = synth.water_run(walkers_per_stage=2, n_bins=10)
    st = synth.initial_state(sp, run, lam0=[0.2, 0.4, 0.6, 0.8])
    e1, _ = make_engine(sp, run, state=st, graph_steps=4)
    for w in range(run.n_walkers):
        g, ref = check_forces(e1, sp, st, w)
        assert g["dUdl"] == 0.0 and ref["dUdl"] == 0.0
    osys = oracle.OracleSystem(sp)
    pairs, kind = e1.get_pairs(0)
    opairs, okind = oracle.pair_set(osys, st.x[0], sp.r_cut + run.skin)
    assert len(pairs) > 0 and np.array_equal(pairs, opairs) and np.array_equal(kind, okind)
    e2, _ = make_engine(sp, run, state=st, graph_steps=4)
    e1.step(30)
    e2.step_plain(30)
    for w in range(run.n_walkers):
        a, b = e1.get_state(w), e2.get_state(w)
        assert np.array_equal(a["x"], b["x"]) and a["lam"] == b["lam"]
    for stage in range(2):
        r = e1.read_abf(0, stage)
        assert int(r["count"].sum()) == 2 * 30
        assert np.all(r["sum"] == 0.0) and np.all(r["sumsq"] == 0.0)
