"""The allocation-free entry point la_alch_pairs_static, through the C ABI.

It exists for callers that cannot allocate device memory: code running as a
plugin inside a program that owns the GPU's memory (an MD engine that gives
its force routines fixed buffers), or deployments that must declare their
device footprint up front.  Its scratch is a static device array shared by
all calls, so this file also checks that two calls in a row each start from
a clean scratch.

Reference: the engine's la_energy_forces on the same configuration.  At
lambda = 0 every alchemical pair term vanishes, so the engine's alchemical
forces are F(lambda) - F(0); dU/dlambda and the two alchemical energy terms
are compared directly.  Tolerances are the parity tests': 1e-5 relative.
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
    out = torch.empty(5, dtype=torch.float64, device=dev)

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
