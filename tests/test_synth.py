"""The seeded synthetic inputs match the recipe they are documented with:
counts, box edges and densities, molecule geometry, parameter ranges,
neutrality, no overlapping atoms, and determinism per seed (CPU only)."""
import numpy as np
import pytest

from paper_2307_08006_gb300 import synth


def min_image(d, box):
    return d - box * np.round(d / box)


def min_pair_distance(x, box, skip_same=None):
    """Smallest periodic distance between atoms (optionally ignoring pairs
    that share a group id)."""
    from scipy.spatial import cKDTree

    tree = cKDTree(np.mod(x, box), boxsize=box)
    pairs = tree.query_pairs(0.3, output_type="ndarray")
    if skip_same is not None:
        pairs = pairs[skip_same[pairs[:, 0]] != skip_same[pairs[:, 1]]]
    if len(pairs) == 0:
        return np.inf
    d = min_image(x[pairs[:, 0]] - x[pairs[:, 1]], box)
    return float(np.sqrt((d * d).sum(1)).min())


def test_lj_fluid_recipe():
    sp = synth.lj_fluid()
    assert sp.n == 257 and sp.box == pytest.approx((256 / 0.8) ** (1 / 3), rel=1e-12)
    a = sp.box / 4
    np.testing.assert_allclose(sp.x[-1], [a / 2] * 3, rtol=1e-6)
    assert (sp.sigma[-1], sp.epsilon[-1], sp.alch[-1]) == (1.2, 1.5, 1)
    assert sp.alch[:-1].sum() == 0 and np.all(sp.sigma[:-1] == 1.0) and np.all(sp.epsilon[:-1] == 1.0)
    # every lattice atom within the +-0.05 jitter of an FCC site
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    sites = np.array([(np.array([i, j, k]) + b) * a for i in range(4) for j in range(4) for k in range(4)
                      for b in basis])
    d = min_image(sp.x[:-1].astype(np.float64) - sites, sp.box)
    assert np.abs(d).max() <= 0.05 + 1e-6
    assert np.array_equal(synth.lj_fluid().x, sp.x)
    assert not np.array_equal(synth.lj_fluid(seed=1).x, sp.x)


def test_solvation_box_recipe():
    sp = synth.water_box(4096, 12, seed=8007)
    nw = 3 * 4096
    assert sp.n == 12300 and sp.box == pytest.approx(5.0, rel=1e-12)
    assert sp.n / sp.box ** 3 == pytest.approx(98.4, rel=1e-3)
    x = sp.x.astype(np.float64)
    # every water: O-H 0.09572 nm, H-O-H 104.52 degrees (within FP32 storage)
    o, h1, h2 = x[0:nw:3], x[1:nw:3], x[2:nw:3]
    b1, b2 = min_image(h1 - o, sp.box), min_image(h2 - o, sp.box)
    r1, r2 = np.linalg.norm(b1, axis=1), np.linalg.norm(b2, axis=1)
    np.testing.assert_allclose(r1, 0.09572, atol=2e-6)
    np.testing.assert_allclose(r2, 0.09572, atol=2e-6)
    ang = np.degrees(np.arccos((b1 * b2).sum(1) / (r1 * r2)))
    np.testing.assert_allclose(ang, 104.52, atol=5e-3)
    # neutral; solute: 12 alchemical sites, 0.15 nm chain, parameter ranges
    assert abs(sp.charge.sum()) < 1e-9
    sol = slice(nw, sp.n)
    assert np.all(sp.alch[sol] == 1) and sp.alch[:nw].sum() == 0
    assert np.all((sp.sigma[sol] >= 0.3) & (sp.sigma[sol] <= 0.4))
    assert np.all((sp.epsilon[sol] >= 0.2) & (sp.epsilon[sol] <= 0.6))
    steps = np.linalg.norm(min_image(np.diff(x[sol], axis=0), sp.box), axis=1)
    np.testing.assert_allclose(steps, 0.15, atol=2e-6)
    # topology: two bonds and one angle per water, 11 chain bonds; one
    # exclusion group per molecule
    assert len(sp.bond_ij) == 2 * 4096 + 11 and len(sp.angle_ijk) == 4096
    assert np.array_equal(sp.excl_group[:nw], np.repeat(np.arange(4096), 3))
    assert np.all(sp.excl_group[sol] == 4096)
    # no two molecules closer than 0.15 nm (the lattice start is not overlapped;
    # the closest contacts are solute sites and water hydrogens, 0.16 nm)
    assert min_pair_distance(x, sp.box, skip_same=sp.excl_group) > 0.15


def test_uneven_batch_recipe():
    specs = synth.uneven_batch()
    assert [s.n for s in specs] == [3 * w + s for w, s in zip(synth.UNEVEN_WATERS, synth.UNEVEN_SOLUTES)]
    run = synth.uneven_run()
    for s, nw in zip(specs, synth.UNEVEN_WATERS):
        assert s.box == pytest.approx((nw / 32.768) ** (1 / 3), rel=1e-12)  # the 4096-water density
        assert s.box >= 2 * (s.r_cut + run.skin)
        assert s.r_cut == (0.85 if nw == 256 else 1.0)
        assert abs(s.charge.sum()) < 1e-9
    assert run.n_walkers == 8 and len(specs) * run.n_walkers == 64


@pytest.mark.slow
def test_large_complex_recipe():
    sp = synth.large_complex()
    nw = 3 * 31000
    assert sp.n == 96040 and sp.n / sp.box ** 3 == pytest.approx(98.4, rel=1e-9)
    assert len(sp.posres_idx) == 3000 and sp.posres_k == 1000.0
    assert np.array_equal(sp.posres_idx, nw + np.arange(3000))
    assert np.all(sp.alch[nw + 3000:] == 1) and sp.alch[:nw + 3000].sum() == 0
    assert len(sp.fb_a) == 40 and len(sp.fb_b) > 0 and sp.fb_d0 == 1.0 and sp.fb_k == 1000.0
    assert np.all(sp.fb_b >= nw) and np.all(sp.fb_b < nw + 3000)
    # chain 1-2 and 1-3 exclusions of the chain sites
    c = nw + 10
    assert sorted(sp.excl_extra[c]) == [c - 2, c - 1, c + 1, c + 2]
    # waters keep their distance from the chain and the ligand
    x = sp.x.astype(np.float64)
    from scipy.spatial import cKDTree

    tree = cKDTree(np.mod(x[nw:], sp.box), boxsize=sp.box)
    dist, _ = tree.query(np.mod(x[0:nw:3], sp.box), k=1)
    assert dist.min() > 0.33 - 2 * np.sqrt(3) * 0.005


def test_run_parameters():
    run = synth.water_run()
    assert run.kT == pytest.approx(0.0083144626 * 300.0, rel=1e-12)
    assert run.m_lambda == pytest.approx(0.6276, rel=1e-12)  # 150000 kcal/mol fs^2 (Sec. 2.2)
    assert run.gamma_lambda == 1000.0 and run.dt == 0.001 and run.n_walkers == 16
    assert [(s.lo, s.hi, s.n_bins) for s in run.stages] == [(0.0, 0.5, 100), (0.5, 1.0, 100)]


def test_initial_state_maxwell_boltzmann():
    sp = synth.water_box(4096, 12, seed=8007)
    run = synth.water_run()
    st = synth.initial_state(sp, run)
    assert st.x.shape == (16, sp.n, 3) and np.array_equal(st.x[3], sp.x)
    # per component <m v^2> = kT, over 16 x 12300 x 3 samples
    mv2 = (sp.mass[None, :, None] * st.v.astype(np.float64) ** 2).mean()
    assert mv2 == pytest.approx(run.kT, rel=0.01)
    # lambda at each stage's lower wall
    assert np.array_equal(st.lam, np.repeat([0.0, 0.5], 8))
    st2 = synth.initial_state(sp, run)
    assert np.array_equal(st.v, st2.v) and np.array_equal(st.plam, st2.plam)
