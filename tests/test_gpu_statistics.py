"""Statistical and per-bin parity of the free-energy read-outs on the GPU.

- Delta A of the two-stage water path (vdW stage with soft-core LJ on
  [0, 0.5], Coulomb stage with lambda_e scaling of the reaction field on
  [0.5, 1]; SI Table S1 staging, Sec. 2.3 Riemann-sum TI) from GPU and oracle
  runs of the 256-water system agrees within two combined standard errors,
  per stage and summed.
- The theta statistics of dDeltaA/dtheta for the solute's (epsilon, sigma,
  q) (la_read_theta) equal the oracle's accumulators bin by bin on a short
  seeded run (same Philox streams), and so does the derivative.
- dDeltaA/dk1 of the lambda-switched harmonic well by both estimators, the
  TI bin estimator sum_k w [<d2U/dl dth>_k - Cov_k(dU/dl, dU/dth)/kT] and the
  end-point difference <dU/dth>_(lambda=1) - <dU/dth>_(lambda=0) (fixed-lambda
  runs), against the closed form d kT / (2 k1), on the GPU and the oracle.
Oracle values come from oracle/ only.
"""
import numpy as np
import pytest

import oracle
from paper_2307_08006_gb300 import labf, synth

pytestmark = pytest.mark.gpu


def _water256():
    sp = synth.water_box(256, 4, seed=720, r_cut=0.85)
    rng = np.random.default_rng(720)
    sp.x = ((sp.x + rng.normal(0.0, 0.01, sp.x.shape)) % sp.box).astype(np.float32)
    return sp


def _water_run(seed, wps=4, n_bins=5, steps_lam=None):
    run = synth.water_run(seed=seed, walkers_per_stage=wps, n_bins=n_bins, n_full=50.0)
    run.gamma_lambda = 100.0  # faster lambda diffusion for a short test run
    lam0 = list(np.linspace(0.05, 0.45, wps)) + list(np.linspace(0.55, 0.95, wps))
    return run, lam0


@pytest.mark.slow
def test_water_two_stage_delta_a_gpu_vs_oracle_two_combined_se():
    sp = _water256()
    oracle.set_threads(8)
    steps, seeds = 1500, range(6)
    res = {"gpu": [], "cpu": []}
    for seed in seeds:
        run, lam0 = _water_run(730 + seed)
        st = synth.initial_state(sp, run, lam0=lam0)
        eng = labf.engine_for(sp, run, st)
        eng.step(steps)
        g = [eng.read_abf(0, k) for k in range(2)]
        assert not any(r["empty_bin"] for r in g)
        res["gpu"].append([g[0]["dA"], g[1]["dA"]])
        eng.close()
        sim = oracle.Simulation(sp, run, st)
        sim.run(steps)
        c = [sim.delta_a(k)[2] for k in range(2)]
        assert np.all(np.isfinite(c))
        res["cpu"].append(c)
    g, c = np.asarray(res["gpu"]), np.asarray(res["cpu"])
    g = np.column_stack([g, g.sum(1)])
    c = np.column_stack([c, c.sum(1)])
    for k, name in enumerate(("vdW stage", "Coulomb stage", "sum")):
        se = np.sqrt(g[:, k].var(ddof=1) / len(g) + c[:, k].var(ddof=1) / len(c))
        assert abs(g[:, k].mean() - c[:, k].mean()) <= 2.0 * se + 1e-9, (name, g[:, k], c[:, k], se)


def test_theta_statistics_match_oracle_bin_by_bin():
    sp = synth.water_box(100, 6, seed=31, box=1.5, r_cut=0.6)
    rng = np.random.default_rng(31)
    sp.x = ((sp.x + rng.normal(0.0, 0.01, sp.x.shape)) % sp.box).astype(np.float32)
    run = synth.water_run(seed=33, walkers_per_stage=2, n_bins=2)
    run.theta_stats = True
    st = synth.initial_state(sp, run, lam0=[0.1, 0.3, 0.6, 0.8])
    eng = labf.engine_for(sp, run, st)
    sim = oracle.Simulation(sp, run, st)
    eng.step(6)
    sim.run(6)
    P = 3 * sp.n_alch + 1
    for stage in range(2):
        g = eng.read_theta(0, stage)
        o0, o1 = sim.stage_off[stage], sim.stage_off[stage + 1]
        for key, okey in (("sum_d2", "th_d2"), ("sum_d", "th_d"), ("sum_sd", "th_sd")):
            ref = sim.a[okey][o0:o1, :P]
            scale = max(1.0, float(np.abs(ref).max()))
            np.testing.assert_allclose(g[key][:, :3 * sp.n_alch], ref[:, :3 * sp.n_alch], rtol=2e-4,
                                       atol=2e-5 * scale, err_msg=f"{key} stage {stage}")
        ref = sim.theta_gradient(stage)[:3 * sp.n_alch]
        assert not g["empty_bin"]
        np.testing.assert_allclose(g["dA_dtheta"][:3 * sp.n_alch], ref, rtol=2e-3,
                                   atol=2e-4 * max(1.0, float(np.abs(ref).max())))


def _endpoint_run(seed):
    """Two frozen walkers per end point: lambda = 0 and lambda = 1 (one stage
    of two bins, bias off, theta statistics on)."""
    run = synth.harmonic_run(seed=seed, n_walkers=4, n_bins=2)
    run.lambda_dynamics = False
    run.abf_on = False
    run.theta_stats = True
    return run, [0.0, 0.0, 1.0, 1.0]


def test_theta_gradient_both_estimators_closed_form_gpu_and_oracle():
    sp = synth.harmonic_well(dims=1, k0=1.0, k1=4.0)
    exact = 1.0 / (2.0 * 4.0)  # d kT / (2 k1) with d = 1, kT = 1
    # TI bin estimator (lambda-ABF on [0, 1])
    ti = []
    for seed in (331, 332, 333):
        run = synth.harmonic_run(seed=seed, n_walkers=4)
        run.theta_stats = True
        eng = labf.engine_for(sp, run)
        eng.step(200_000)
        ti.append(eng.read_theta(0, 0)["dA_dtheta"][-1])
        eng.close()
    ti_gpu = float(np.mean(ti))
    # end-point estimator: <dU/dk1> at lambda = 1 minus at lambda = 0
    erun, lam0 = _endpoint_run(334)
    st = synth.initial_state(sp, erun, lam0=lam0)
    e2 = labf.engine_for(sp, erun, st)
    e2.step(200_000)
    th = e2.read_theta(0, 0)
    cnt = e2.read_abf(0, 0)["count"]
    mean_d = th["sum_d"][:, -1] / cnt
    ep_gpu = mean_d[1] - mean_d[0]
    sim = oracle.Simulation(sp, erun, st)
    sim.run(50_000)
    _, _, c = sim.stage_bins(0)
    md = sim.a["th_d"][0:2, -1] / c
    ep_cpu = md[1] - md[0]
    assert mean_d[0] == 0.0 and md[0] == 0.0  # dU/dk1 = lambda x^2 / 2 vanishes at lambda = 0
    assert ti_gpu == pytest.approx(exact, abs=0.02)
    assert ep_gpu == pytest.approx(exact, abs=0.01)
    assert ep_cpu == pytest.approx(exact, abs=0.015)
    assert abs(ti_gpu - ep_gpu) < 0.025


def test_mass_friction_sweep_driver_runs():
    """The lambda mass / friction sweep (SI S2) on the 256-water two-stage
    system, short: every (mass, friction, seed) system advances, lambda moves,
    and Delta A is finite wherever every bin has samples."""
    from paper_2307_08006_gb300 import compare

    m0 = synth.M_LAMBDA_KJ_PS2
    rows = compare.sweep(3000, [1, 2], [m0 / 10, m0], [100.0], every=1000)
    assert len(rows) == 2
    for r in rows:
        assert r["seeds"] == 2 and np.isfinite(r["lambda_span"]) and r["lambda_span"] > 0.0
        if r["dA_mean"] is not None:
            assert np.isfinite(r["dA_mean"])
    # the lighter lambda particle moves further in the same time
    assert rows[0]["lambda_span"] > rows[1]["lambda_span"]
