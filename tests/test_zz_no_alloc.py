"""The allocation-free entry point la_alch_pairs_static, through the C ABI.

It exists for callers that cannot allocate device memory: code running as a
plugin inside a program that owns the GPU's memory (an MD engine that gives
its force routines fixed buffers), or deployments that must declare their
device footprint up front.  Its scratch is a static device array shared by
all calls, so this file also checks that two calls in a row each start from
a clean scratch.

References: the engine's la_energy_forces on the same configuration, and
the FP64 oracle.  At lambda = 0 every alchemical pair term vanishes
(lambda_v = lambda_e = 0), so the alchemical forces are F(lambda) - F(0) of
either; dU/dlambda and the two alchemical energy terms are compared
directly.  Tolerances are the parity tests': 1e-5 relative.
"""
import numpy as np
import pytest

from paper_2307_08006_gb300 import labf, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _system():
    sp = synth.water_box(100, 6, seed=41, box=1.5, r_cut=0.6)
    rng = np.random.default_rng(41)
    sp.x = ((sp.x + rng.normal(0.0, 0.01, sp.x.shape)) % sp.box).astype(np.float32)
    run = synth.water_run(seed=42, walkers_per_stage=1, n_bins=10)
    return sp, run


def test_static_entry_matches_engine_on_two_calls():
    import torch

    sp, run = _system()
    state = synth.initial_state(sp, run, lam0=[0.3, 0.7])
    eng = labf.engine_for(sp, run, state)
    dev = torch.device("cuda", 0)
    x = torch.tensor(eng.get_state(0)["x"], device=dev)
    assert np.array_equal(eng.get_state(1)["x"], x.cpu().numpy())
    t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    q, sig, eps = t(sp.charge, torch.float32), t(sp.sigma, torch.float32), t(sp.epsilon, torch.float32)
    alch, grp = t(sp.alch, torch.uint8), t(sp.excl_group, torch.int32)
    alch_idx = t(np.nonzero(sp.alch)[0], torch.int32)
    forces = torch.empty((sp.n, 3), dtype=torch.float32, device=dev)
    out = torch.empty(6, dtype=torch.float64, device=dev)

    # engine reference: alchemical forces = F(lambda) - F(0) (walker 0 at lambda = 0)
    eng.set_state(0, lam=0.0)
    f0 = eng.energy_forces(0)["F"].cpu().numpy().astype(np.float64)
    for walker, lam in ((0, 0.3), (1, 0.7)):  # two calls in a row, same scratch
        eng.set_state(walker, lam=lam)
        ref = eng.energy_forces(walker)
        labf.alch_pairs_static(x, q, sig, eps, alch, grp, alch_idx, sp.box, sp.r_cut, sp.eps_rf, sp.coul,
                               lam, sp.b_v, sp.b_e, sp.sc_alpha, sp.sc_n, sp.sc_m, forces=forces, out=out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert o[5] == 0.0, f"device status {int(o[5]):#x}"
        f = forces.cpu().numpy().astype(np.float64)
        fref = ref["F"].cpu().numpy().astype(np.float64)
        scale = max(1.0, abs(o[1]) + abs(o[2]))
        assert abs(o[0] - ref["dUdl"]) <= TOL * scale, (lam, o[0], ref["dUdl"])
        assert o[3] == pytest.approx(ref["terms"][2], rel=TOL, abs=TOL)
        assert o[4] == pytest.approx(ref["terms"][3], rel=TOL, abs=TOL)
        err = np.sqrt(((f - (fref - f0)) ** 2).sum() / (fref ** 2).sum())
        assert err < TOL, (lam, err)
        assert np.abs(f).max() > 0.0
    eng.close()


def test_static_entry_rejects_sizes_beyond_its_scratch():
    import torch

    dev = torch.device("cuda", 0)
    n = 131072 + 1  # one atom beyond LA_STATIC_MAX_ATOMS
    x = torch.zeros((n, 3), dtype=torch.float32, device=dev)
    z = torch.zeros(n, dtype=torch.float32, device=dev)
    a = torch.zeros(n, dtype=torch.uint8, device=dev)
    g = torch.full((n,), -1, dtype=torch.int32, device=dev)
    idx = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(labf.LabfError, match="static scratch"):
        labf.alch_pairs_static(x, z, z, z, a, g, idx, 100.0, 1.0, 78.0, 1.0, 0.5, 0.5, 0.5)


def test_static_entry_matches_oracle():
    """The static entry point against the FP64 oracle directly: the oracle's
    alchemical forces F(lambda) - F(0), dU/dlambda, dU/dlambda_v,
    dU/dlambda_e and the soft-core LJ and scaled RF energies, at lambdas on
    both stages, on the kinks b_v = b_e = 0.5 and at the ends, also with
    soft-core powers n = m = 2."""
    import torch

    import oracle

    sp, _ = _system()
    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    x = t(sp.x, torch.float32)
    q, sig, eps = t(sp.charge, torch.float32), t(sp.sigma, torch.float32), t(sp.epsilon, torch.float32)
    alch, grp = t(sp.alch, torch.uint8), t(sp.excl_group, torch.int32)
    alch_idx = t(np.nonzero(sp.alch)[0], torch.int32)
    for n_, m_ in ((1, 1), (2, 2)):
        spx = synth.with_changes(sp, sc_n=n_, sc_m=m_)
        osys = oracle.OracleSystem(spx)
        x64 = sp.x.astype(np.float64)
        f0 = oracle.energy_forces(osys, x64, 0.0)["F"]
        for lam in (0.0, 0.2, 0.5, 0.8, 1.0):
            ref = oracle.energy_forces(osys, x64, lam)
            forces, out = labf.alch_pairs_static(x, q, sig, eps, alch, grp, alch_idx, sp.box, sp.r_cut, sp.eps_rf,
                                                 sp.coul, lam, sp.b_v, sp.b_e, sp.sc_alpha, n_, m_)
            torch.cuda.synchronize()
            o = out.cpu().numpy()
            assert o[5] == 0.0
            scale = max(1.0, abs(ref["dl"][0]) + abs(ref["dl"][1]))
            assert abs(o[0] - ref["dUdl"]) <= TOL * scale, (n_, lam, o[0], ref["dUdl"])
            assert abs(o[1] - ref["dl"][0]) <= TOL * scale, (n_, lam, o[1], ref["dl"][0])
            assert abs(o[2] - ref["dl"][1]) <= TOL * scale, (n_, lam, o[2], ref["dl"][1])
            escale = max(1.0, abs(ref["terms"][2]) + abs(ref["terms"][3]))
            assert abs(o[3] - ref["terms"][2]) <= TOL * escale
            assert abs(o[4] - ref["terms"][3]) <= TOL * escale
            fa = ref["F"] - f0
            f = forces.cpu().numpy().astype(np.float64)
            if lam == 0.0:
                assert np.abs(f).max() == 0.0
            else:
                err = np.sqrt(((f - fa) ** 2).sum() / (fa ** 2).sum())
                assert err < TOL, (n_, lam, err)


def test_static_entry_reports_bad_index_and_nonfinite():
    """Device-side problems come back in out[5] as LA_STATUS_* bits, without
    a fault: an alchemical index that names a non-alchemical atom, and a NaN
    coordinate."""
    import torch

    sp, _ = _system()
    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    q, sig, eps = t(sp.charge, torch.float32), t(sp.sigma, torch.float32), t(sp.epsilon, torch.float32)
    alch, grp = t(sp.alch, torch.uint8), t(sp.excl_group, torch.int32)
    bad = t(np.array([0], np.int32) if not sp.alch[0] else np.array([1], np.int32), torch.int32)
    x = t(sp.x, torch.float32)
    _, out = labf.alch_pairs_static(x, q, sig, eps, alch, grp, bad, sp.box, sp.r_cut, sp.eps_rf, sp.coul, 0.5,
                                    sp.b_v, sp.b_e)
    torch.cuda.synchronize()
    assert int(out[5].item()) & 0x20
    xn = sp.x.copy()
    xn[int(np.nonzero(~sp.alch.astype(bool))[0][0])] = np.nan
    idx = t(np.nonzero(sp.alch)[0], torch.int32)
    _, out = labf.alch_pairs_static(t(xn, torch.float32), q, sig, eps, alch, grp, idx, sp.box, sp.r_cut, sp.eps_rf,
                                    sp.coul, 0.5, sp.b_v, sp.b_e)
    torch.cuda.synchronize()
    assert int(out[5].item()) & 0x2
    # a clean call afterwards starts from a cleared status word
    _, out = labf.alch_pairs_static(x, q, sig, eps, alch, grp, idx, sp.box, sp.r_cut, sp.eps_rf, sp.coul, 0.5,
                                    sp.b_v, sp.b_e)
    torch.cuda.synchronize()
    assert out[5].item() == 0.0
