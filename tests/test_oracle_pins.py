"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values
printed in the paper (SI Table S1), published known-answer vectors
(Philox), textbook special cases (plain LJ, shifted Coulomb), closed forms
(RF zero at the cutoff, BAOAB's exact harmonic variance, the free energy of
a lambda-switched harmonic well), finite differences, invariants (Newton's
third law, translation invariance) and constructed boundary cases of the
integer pair set.
"""
import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_2307_08006_gb300 import synth


# ----------------------------------------------------------------------------
# lambda path: SI Table S1 and Sec. 3.1.1
# ----------------------------------------------------------------------------
def test_lambda_schedule_matches_table_s1():
    rows = read_golden("lambda_schedule_tableS1.txt")
    assert len(rows) == 24
    for lam, le, lv in rows:
        out = oracle.lambda_path(float(lam), 0.5, 0.5)
        assert out[0] == pytest.approx(float(lv), abs=1e-12)
        assert out[1] == pytest.approx(float(le), abs=1e-12)


def test_lambda_path_slopes_and_endpoints():
    # no interactions at lambda = 0 and full interactions at lambda = 1 (Sec. 3.1.1)
    for bv, be in ((0.5, 0.5), (1.0, 0.5), (0.7, 0.2)):
        assert tuple(oracle.lambda_path(0.0, bv, be)[:2]) == (0.0, 0.0)
        assert tuple(oracle.lambda_path(1.0, bv, be)[:2]) == (1.0, 1.0)
        for lam in np.linspace(0.013, 0.987, 17):
            h = 1e-7
            if abs(lam - bv) < 1e-3 or abs(lam - be) < 1e-3:
                continue
            p, m = oracle.lambda_path(lam + h, bv, be), oracle.lambda_path(lam - h, bv, be)
            d = oracle.lambda_path(lam, bv, be)
            assert d[2] == pytest.approx((p[0] - m[0]) / (2 * h), rel=1e-6, abs=1e-9)
            assert d[3] == pytest.approx((p[1] - m[1]) / (2 * h), rel=1e-6, abs=1e-9)
    # one-sided slopes at the kinks
    assert oracle.lambda_path(0.5, 0.5, 0.5)[2] == 0.0
    assert oracle.lambda_path(0.5, 0.5, 0.5)[3] == 0.0


# ----------------------------------------------------------------------------
# Philox4x32-10 and the normals drawn from it
# ----------------------------------------------------------------------------
def test_philox_known_answers():
    for row in read_golden("philox4x32_10_kat.txt"):
        v = [int(t, 16) for t in row]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_normals_moments():
    z = np.concatenate([oracle.normals4(7, 3, s, i, 0) for s in range(50) for i in range(1000)])
    n = z.size
    assert abs(z.mean()) < 5.0 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert abs(np.mean(z ** 3)) < 5.0 * np.sqrt(15.0 / n)
    assert abs(np.mean(z ** 4) - 3.0) < 5.0 * np.sqrt(96.0 / n)
    # different tags, walkers and steps give different streams
    a = oracle.normals4(7, 3, 5, 11, 0)
    assert not np.allclose(a, oracle.normals4(7, 3, 5, 11, 1))
    assert not np.allclose(a, oracle.normals4(7, 4, 5, 11, 0))
    assert not np.allclose(a, oracle.normals4(7, 3, 6, 11, 0))


# ----------------------------------------------------------------------------
# pair potentials: textbook special cases and closed forms
# ----------------------------------------------------------------------------
def _two_atoms(r, q=(0.0, 0.0), alch=(0, 0), sig=(1.0, 1.0), eps=(1.0, 1.0), rc=2.5, eps_rf=78.0,
               coul=1.0, bv=1.0, be=0.0, alpha=0.5, box=20.0):
    x = np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]], np.float32)
    return synth.SystemSpec(
        name="pair", box=box, mass=np.ones(2), charge=np.asarray(q, float),
        sigma=np.asarray(sig, float), epsilon=np.asarray(eps, float),
        alch=np.asarray(alch, np.uint8), excl_group=np.full(2, -1, np.int32),
        excl_extra=np.full((2, 4), -1, np.int32), x=x, r_cut=rc, eps_rf=eps_rf, coul=coul,
        b_v=bv, b_e=be, sc_alpha=alpha)


def _lj_textbook(r, sig, eps):
    return 4.0 * eps * ((sig / r) ** 12 - (sig / r) ** 6)


def test_softcore_reduces_to_textbook_lj_at_full_coupling():
    for r in (0.95, 1.1, 1.5, 2.2):
        sp = _two_atoms(r, alch=(1, 0), sig=(1.2, 1.0), eps=(1.5, 1.0))
        o = oracle.OracleSystem(sp)
        xr = sp.x.astype(np.float64)
        res = oracle.energy_forces(o, xr, 1.0)
        r_act = float(xr[1, 0] - xr[0, 0])
        ref = _lj_textbook(r_act, 1.1, np.sqrt(1.5))
        assert res["terms"][2] == pytest.approx(ref, rel=1e-12)
        # the same pair as a normal pair (no alchemical atom)
        sp2 = _two_atoms(r, sig=(1.2, 1.0), eps=(1.5, 1.0))
        res2 = oracle.energy_forces(oracle.OracleSystem(sp2), xr, 1.0)
        assert res2["terms"][0] == pytest.approx(ref, rel=1e-12)
        np.testing.assert_allclose(res["F"], res2["F"], rtol=1e-12, atol=1e-14)


def test_softcore_vanishes_at_zero_coupling():
    sp = synth.lj_fluid()
    o = oracle.OracleSystem(sp)
    x = sp.x.astype(np.float64)
    r0 = oracle.energy_forces(o, x, 0.0)
    assert r0["terms"][2] == 0.0 and r0["terms"][3] == 0.0
    assert np.all(r0["F"][-1] == 0.0)
    # the solvent feels nothing from the decoupled solute: same forces as a
    # system where the solute is far away (beyond the cutoff of every atom)
    sp_far = synth.with_changes(sp, epsilon=np.concatenate([sp.epsilon[:-1], [0.0]]))
    rf = oracle.energy_forces(oracle.OracleSystem(sp_far), x, 1.0)
    np.testing.assert_allclose(r0["F"][:-1], rf["F"][:-1], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n,m", [(1, 1), (2, 1), (1, 2), (2, 2)])
def test_softcore_finite_at_overlap(n, m):
    # at lambda_v < 1 the soft-core energy stays finite at r = 0 (Sec. 3.1.2):
    # with sigma = eps = 1 it tends to lambda^n 4 (1/s^2 - 1/s), s = alpha (1-lambda)^m
    for lv in (0.1, 0.5, 0.9):
        sp = synth.with_changes(_two_atoms(1e-4, alch=(1, 0)), sc_n=n, sc_m=m)
        o = oracle.OracleSystem(sp)
        res = oracle.energy_forces(o, sp.x.astype(np.float64), lv)
        alpha = 0.5
        s = alpha * (1 - lv) ** m
        assert res["terms"][2] == pytest.approx(lv ** n * 4 * (1 / s ** 2 - 1 / s), rel=1e-6)


def _bare(n, x, box=3.0, mass=None, group=None, **kw):
    """n uncharged atoms with no Lennard-Jones interaction."""
    return synth.SystemSpec(
        name="bare", box=box, mass=np.ones(n) if mass is None else np.asarray(mass, float),
        charge=np.zeros(n), sigma=np.zeros(n), epsilon=np.zeros(n), alch=np.zeros(n, np.uint8),
        excl_group=np.full(n, -1, np.int32) if group is None else np.asarray(group, np.int32),
        excl_extra=np.full((n, 4), -1, np.int32), x=np.asarray(x, np.float32), **kw)


@pytest.mark.parametrize("origin", [(1.5, 1.5, 1.5), (2.97, 0.02, 1.0)])
def test_bonded_terms_closed_form(origin):
    """A water built with O-H lengths r0 + 0.004 and r0 - 0.003 and an
    H-O-H angle theta0 + 0.05 rad (second case: the molecule straddles two
    box faces): U_bond = 1/2 k_b (0.004^2 + 0.003^2), U_angle = 1/2 k_t 0.05^2."""
    L, r0, t0, kb, kt = 3.0, 0.09572, np.deg2rad(104.52), 502416.0, 628.02
    o = np.array(origin)
    th = t0 + 0.05
    x = np.array([o, o + (r0 + 0.004) * np.array([1.0, 0.0, 0.0]),
                  o + (r0 - 0.003) * np.array([np.cos(th), -np.sin(th), 0.0])]) % L
    sp = _bare(3, x, box=L, group=[0, 0, 0], bond_ij=np.array([[0, 1], [0, 2]], np.int32),
               bond_r0=np.full(2, r0), bond_k=np.full(2, kb), angle_ijk=np.array([[1, 0, 2]], np.int32),
               angle_t0=np.array([t0]), angle_k=np.array([kt]))
    res = oracle.energy_forces(oracle.OracleSystem(sp), x, 1.0)
    assert res["terms"][4] == pytest.approx(0.5 * kb * (0.004 ** 2 + 0.003 ** 2), rel=1e-9)
    assert res["terms"][5] == pytest.approx(0.5 * kt * 0.05 ** 2, rel=1e-9)
    assert np.all(res["terms"][[0, 1, 2, 3, 6]] == 0.0)
    np.testing.assert_allclose(res["F"].sum(axis=0), 0.0, atol=1e-7)  # internal forces


def test_restraint_terms_closed_form():
    """Positional restraint across a box face, flat-bottom restraint on two
    centres of mass (outside and inside d0) and the lambda-switched well with
    its dU/dlambda, each against its closed form."""
    L = 3.0
    # positional: displacement (0.03, -0.04, 0.012) from a reference just
    # inside the upper face, the atom wrapped to the lower side
    x0 = np.array([[2.99, 1.0, 0.005]])
    x = (x0 + [0.03, -0.04, 0.012]) % L
    sp = _bare(1, x, box=L, posres_idx=np.array([0], np.int32), posres_x0=x0, posres_k=1000.0)
    res = oracle.energy_forces(oracle.OracleSystem(sp), x, 0.3)
    assert res["terms"][6] == pytest.approx(500.0 * (0.03 ** 2 + 0.04 ** 2 + 0.012 ** 2), rel=1e-9)
    np.testing.assert_allclose(res["F"][0], [-30.0, 40.0, -12.0], rtol=1e-9)
    # flat bottom: group A = masses 1 and 3 (centre a quarter of the way from
    # atom 0 to atom 1), group B = one atom; centre distance d0 + 0.02 / d0 - 0.02
    d0, k = 1.0, 800.0
    for ex, expect in ((0.02, 0.5 * k * 0.02 ** 2), (-0.02, 0.0)):
        a0 = np.array([0.5, 1.0, 1.0])
        a1 = a0 + [0.4, 0.0, 0.0]
        com = a0 + 0.75 * (a1 - a0)
        b = com + (d0 + ex) * np.array([0.0, 0.6, 0.8])
        x = np.array([a0, a1, b])
        sp = _bare(3, x, box=L, mass=[1.0, 3.0, 2.0], fb_a=np.array([0, 1], np.int32),
                   fb_b=np.array([2], np.int32), fb_d0=d0, fb_k=k)
        res = oracle.energy_forces(oracle.OracleSystem(sp), x, 0.5)
        assert res["terms"][6] == pytest.approx(expect, rel=1e-9, abs=1e-15)
        np.testing.assert_allclose(res["F"].sum(axis=0), 0.0, atol=1e-9)
    # lambda-switched well: U = 1/2 ((1 - lambda) k0 + lambda k1) r^2 with r^2 = 0.09
    x0 = np.array([[1.0, 1.0, 1.0]])
    x = x0 + [0.1, 0.2, -0.2]
    sp = _bare(1, x, box=L, lh_idx=np.array([0], np.int32), lh_x0=x0, lh_k0=100.0, lh_k1=400.0, lh_dims=3)
    for lam in (0.0, 0.25, 1.0):
        res = oracle.energy_forces(oracle.OracleSystem(sp), x, lam)
        kl = (1 - lam) * 100.0 + lam * 400.0
        assert res["terms"][6] == pytest.approx(0.5 * kl * 0.09, rel=1e-9)
        assert res["dUdl"] == pytest.approx(0.5 * 300.0 * 0.09, rel=1e-9)


def test_reaction_field_closed_forms():
    rc = 1.2
    # U(r_c) = 0 for any eps_rf
    for eps_rf in (1.0, 4.0, 78.0, 0.0):
        sp = _two_atoms(rc * (1 - 1e-9), q=(0.5, -0.7), sig=(0, 0), eps=(0, 0), rc=rc, eps_rf=eps_rf)
        res = oracle.energy_forces(oracle.OracleSystem(sp), sp.x.astype(np.float64), 1.0)
        assert abs(res["terms"][1]) < 1e-7
    # conducting continuum: the force also vanishes at the cutoff
    r = rc * (1 - 1e-7)
    sp = _two_atoms(r, q=(0.5, -0.7), sig=(0, 0), eps=(0, 0), rc=rc, eps_rf=0.0)
    xs = sp.x.astype(np.float64)
    xs[1, 0] = xs[0, 0] + r
    res = oracle.energy_forces(oracle.OracleSystem(sp), xs, 1.0)
    assert np.abs(res["F"]).max() < 1e-5
    # eps_rf = 1 is a cut-off Coulomb shifted to zero at r_c
    for r in (0.3, 0.7, 1.1):
        sp = _two_atoms(r, q=(0.5, -0.7), sig=(0, 0), eps=(0, 0), rc=rc, eps_rf=1.0, coul=138.935458)
        xs = sp.x.astype(np.float64)
        xs[1, 0] = xs[0, 0] + r
        res = oracle.energy_forces(oracle.OracleSystem(sp), xs, 1.0)
        assert res["terms"][1] == pytest.approx(138.935458 * 0.5 * -0.7 * (1 / r - 1 / rc), rel=1e-12)
        assert res["F"][1, 0] == pytest.approx(138.935458 * 0.5 * -0.7 / r ** 2, rel=1e-12)


@pytest.mark.parametrize("lam", [0.55, 0.8, 1.0])
def test_alchemical_rf_scales_linearly(lam):
    """A pair with one alchemical atom carries lambda_e times the
    reaction-field energy of the same pair as a normal pair (Sec. 3.1.2), and
    its dU/dlambda is dlambda_e/dlambda = 1/(1 - b_e) times that energy."""
    for r in (0.3, 0.7, 1.1):
        kw = dict(q=(0.5, -0.7), sig=(0.0, 0.0), eps=(0.0, 0.0), rc=1.2, bv=0.5, be=0.5)
        alch = oracle.energy_forces(oracle.OracleSystem(_two_atoms(r, alch=(1, 0), **kw)),
                                    _two_atoms(r, **kw).x.astype(np.float64), lam)
        norm = oracle.energy_forces(oracle.OracleSystem(_two_atoms(r, **kw)),
                                    _two_atoms(r, **kw).x.astype(np.float64), lam)
        le = (lam - 0.5) / 0.5
        assert norm["terms"][1] != 0.0
        assert alch["terms"][3] == pytest.approx(le * norm["terms"][1], rel=1e-12)
        assert alch["dUdl"] == pytest.approx(2.0 * norm["terms"][1], rel=1e-12)
        np.testing.assert_allclose(alch["F"], le * norm["F"], rtol=1e-12)


def test_cutoff_truncates():
    sp = _two_atoms(2.6, rc=2.5)
    res = oracle.energy_forces(oracle.OracleSystem(sp), sp.x.astype(np.float64), 1.0)
    assert res["U"] == 0.0 and np.all(res["F"] == 0.0)


# ----------------------------------------------------------------------------
# derivatives against central finite differences
# ----------------------------------------------------------------------------
def _small_water(seed=3):
    sp = synth.water_box(27, 4, seed=seed, box=1.95, r_cut=0.9)
    rng = np.random.default_rng(seed)
    x = (sp.x + rng.normal(0, 0.01, sp.x.shape)).astype(np.float64) % sp.box
    return sp, x


def _restrained_small(seed=4):
    """Small water box whose solute also carries a flat-bottom restraint, a
    lambda-switched well and positional restraints, to exercise every term."""
    sp, x = _small_water(seed)
    n = sp.n
    sp = synth.with_changes(
        sp, posres_idx=np.array([0, 3], np.int32), posres_x0=x[[0, 3]] + 0.05, posres_k=1000.0,
        fb_a=np.arange(n - 4, n, dtype=np.int32), fb_b=np.array([6, 9, 12], np.int32),
        fb_d0=0.05, fb_k=800.0, lh_idx=np.array([n - 1], np.int32), lh_x0=x[[n - 1]] + 0.07,
        lh_k0=100.0, lh_k1=400.0, lh_dims=3, lr_ij=np.array([[n - 3, 9], [2, 20]], np.int32),
        lr_delta=1.2, lr_k=500.0)
    return sp, x


@pytest.mark.parametrize("lam,n,m", [(0.12, 1, 1), (0.37, 1, 1), (0.63, 1, 1), (0.91, 1, 1),
                                     (0.37, 2, 2), (0.63, 2, 1)])
def test_forces_match_finite_differences(lam, n, m):
    sp, x = _restrained_small()
    sp = synth.with_changes(sp, sc_n=n, sc_m=m)
    o = oracle.OracleSystem(sp)
    res = oracle.energy_forces(o, x, lam)
    rng = np.random.default_rng(11)
    h = 1e-6
    for i in list(rng.choice(sp.n, 6, replace=False)) + [sp.n - 1, sp.n - 4]:
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            fd = -(oracle.energy_forces(o, xp, lam)["U"] - oracle.energy_forces(o, xm, lam)["U"]) / (2 * h)
            assert res["F"][i, c] == pytest.approx(fd, rel=2e-5, abs=2e-3)


@pytest.mark.parametrize("lam", [0.05, 0.2, 0.45, 0.55, 0.8, 0.97])
@pytest.mark.parametrize("n,m", [(1, 1), (2, 1), (1, 2), (2, 2)])
def test_dudl_matches_finite_differences(lam, n, m):
    # every soft-core power pair (n, m) of Sec. 3.1.2, not only the default
    sp, x = _restrained_small()
    sp = synth.with_changes(sp, sc_n=n, sc_m=m)
    o = oracle.OracleSystem(sp)
    h = 1e-6
    fd = (oracle.energy_forces(o, x, lam + h)["U"] - oracle.energy_forces(o, x, lam - h)["U"]) / (2 * h)
    assert oracle.energy_forces(o, x, lam)["dUdl"] == pytest.approx(fd, rel=1e-6, abs=1e-4)


@pytest.mark.parametrize("lam,n,m", [(0.2, 1, 1), (0.45, 1, 1), (0.7, 1, 1), (0.45, 2, 2)])
def test_theta_derivatives_match_finite_differences(lam, n, m):
    sp, x = _restrained_small()
    sp = synth.with_changes(sp, sc_n=n, sc_m=m)
    o = oracle.OracleSystem(sp)
    res = oracle.energy_forces(o, x, lam)
    alch = np.nonzero(sp.alch)[0]
    h = 1e-6
    for r, a in enumerate(alch):
        for k, field in enumerate(("epsilon", "sigma", "charge")):
            vals = []
            for sgn in (+1, -1):
                arr = getattr(sp, field).copy()
                arr[a] += sgn * h
                osp = oracle.OracleSystem(synth.with_changes(sp, **{field: arr}))
                e = oracle.energy_forces(osp, x, lam)
                vals.append((e["U"], e["dUdl"]))
            fd_u = (vals[0][0] - vals[1][0]) / (2 * h)
            fd_l = (vals[0][1] - vals[1][1]) / (2 * h)
            assert res["dth"][3 * r + k] == pytest.approx(fd_u, rel=1e-5, abs=1e-3)
            assert res["d2th"][3 * r + k] == pytest.approx(fd_l, rel=1e-5, abs=1e-3)
    # k1 of the lambda-switched well is the last theta entry
    vals = []
    for sgn in (+1, -1):
        osp = oracle.OracleSystem(synth.with_changes(sp, lh_k1=sp.lh_k1 + sgn * 1e-4))
        e = oracle.energy_forces(osp, x, lam)
        vals.append((e["U"], e["dUdl"]))
    assert res["dth"][-1] == pytest.approx((vals[0][0] - vals[1][0]) / 2e-4, rel=1e-6)
    assert res["d2th"][-1] == pytest.approx((vals[0][1] - vals[1][1]) / 2e-4, rel=1e-6)


def test_newton_third_law_and_translation_invariance():
    sp, x = _small_water()
    o = oracle.OracleSystem(sp)
    for lam in (0.3, 0.8):
        res = oracle.energy_forces(o, x, lam)
        tot = res["F"].sum(0)
        assert np.abs(tot).max() < 1e-9 * np.abs(res["F"]).max()
        shifted = (x + np.array([0.37, -1.21, 0.05])) % sp.box
        res2 = oracle.energy_forces(o, shifted, lam)
        assert res2["U"] == pytest.approx(res["U"], rel=1e-10)
        np.testing.assert_allclose(res2["F"], res["F"], rtol=1e-8, atol=1e-8)


# ----------------------------------------------------------------------------
# the integer pair set
# ----------------------------------------------------------------------------
def _brute_pairs(sp, x, r_list):
    """Independent O(N^2) restatement with Python integers."""
    box_inv = 1.0 / sp.box
    u = oracle.quantize(x, box_inv).astype(np.int64)
    R = oracle.list_threshold(r_list, box_inv)
    out = set()
    for i in range(sp.n):
        for j in range(i + 1, sp.n):
            if sp.excl_group[i] >= 0 and sp.excl_group[i] == sp.excl_group[j]:
                continue
            if j in sp.excl_extra[i] or i in sp.excl_extra[j]:
                continue
            if sp.alch[i] and sp.alch[j]:
                continue
            d = [((int(u[i, c]) - int(u[j, c]) + 2 ** 23) % 2 ** 24) - 2 ** 23 for c in range(3)]
            if d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < R:
                out.add((i, j))
    return out


def test_pair_set_matches_brute_force():
    sp, x = _small_water(5)
    o = oracle.OracleSystem(sp)
    pairs, kind = oracle.pair_set(o, x.astype(np.float32), 1.0)
    got = set(map(tuple, pairs.tolist()))
    assert got == _brute_pairs(sp, x.astype(np.float32), 1.0)
    for (i, j), k in zip(pairs.tolist(), kind.tolist()):
        assert k == int(sp.alch[i]) + int(sp.alch[j])


def test_quantize_definition():
    L = 3.0
    xs = np.array([[0.0, 1.5, 2.9999999], [-1e-9, 3.0, 4.5], [-1e-30, 0.75, 0.0]], np.float32)
    u = oracle.quantize(xs, 1.0 / L)
    assert u[0, 0] == 0 and u[0, 1] == 2 ** 23
    assert u[1, 0] == 2 ** 24 - 1  # just below the box origin: the last cell
    assert u[1, 1] == 0  # x = L wraps to 0
    assert u[1, 2] == 2 ** 23
    assert u[2, 0] == 0  # frac of a tiny negative rounds to 1.0, folded to 0
    assert u[2, 1] == 2 ** 22
    assert u.max() < 2 ** 24


def _grid_pair(dx, dy, dz, L=1.0, base=(0, 0, 0)):
    """Two atoms whose quantized coordinates are exact integers."""
    s = 2.0 ** -24
    a = np.array([base], np.float64)
    b = np.array([[(base[0] + dx) % 2 ** 24, (base[1] + dy) % 2 ** 24, (base[2] + dz) % 2 ** 24]])
    x = (np.concatenate([a, b]) * s * L).astype(np.float32)
    return x


def test_pair_set_boundary_ties_and_wrap():
    n = 2
    sp = synth.SystemSpec(name="b", box=1.0, mass=np.ones(n), charge=np.zeros(n),
                          sigma=np.ones(n), epsilon=np.ones(n), alch=np.zeros(n, np.uint8),
                          excl_group=np.full(n, -1, np.int32),
                          excl_extra=np.full((n, 4), -1, np.int32), x=np.zeros((n, 3), np.float32))
    o = oracle.OracleSystem(sp)
    d = 1_000_000  # D = d^2 exactly
    r_list = d * 2.0 ** -24  # R = floor(r_list^2 2^48) = d^2
    assert oracle.list_threshold(r_list, 1.0) == d * d
    # tie D == R: not listed; one unit closer: listed
    assert len(oracle.pair_set(o, _grid_pair(d, 0, 0), r_list)[0]) == 0
    assert len(oracle.pair_set(o, _grid_pair(d - 1, 0, 0), r_list)[0]) == 1
    # across the box edge (minimum image on the 2^24 torus)
    assert len(oracle.pair_set(o, _grid_pair(d - 1, 0, 0, base=(2 ** 24 - 10, 5, 7)), r_list)[0]) == 1
    assert len(oracle.pair_set(o, _grid_pair(-(d - 1), 0, 0, base=(10, 5, 7)), r_list)[0]) == 1
    assert len(oracle.pair_set(o, _grid_pair(-d, 0, 0, base=(10, 5, 7)), r_list)[0]) == 0
    # a diagonal tie: 600^2 + 800^2 = 1000^2
    assert oracle.list_threshold(1000 * 2.0 ** -24, 1.0) == 10 ** 6
    assert len(oracle.pair_set(o, _grid_pair(600, 800, 0), 1000 * 2.0 ** -24)[0]) == 0
    assert len(oracle.pair_set(o, _grid_pair(600, 799, 0), 1000 * 2.0 ** -24)[0]) == 1
    # half a box apart: the torus delta is -2^23 for both orders
    x = _grid_pair(2 ** 23, 0, 0)
    assert len(oracle.pair_set(o, x, 0.5 + 1e-9)[0]) == 1
    assert len(oracle.pair_set(o, x, 0.5)[0]) == 0


def test_pair_set_exclusions():
    sp = synth.water_box(8, 3, seed=2, box=1.2, r_cut=0.5)
    o = oracle.OracleSystem(sp)
    pairs, kind = oracle.pair_set(o, sp.x, 0.59)
    got = set(map(tuple, pairs.tolist()))
    for w in range(8):
        for a in range(3):
            for b in range(a + 1, 3):
                assert (3 * w + a, 3 * w + b) not in got
    sol = range(24, 27)
    for a in sol:
        for b in sol:
            assert (a, b) not in got
    assert set(kind.tolist()) <= {0, 1}
    assert got == _brute_pairs(sp, sp.x, 0.59)


# ----------------------------------------------------------------------------
# integrator and ABF: closed forms and invariants
# ----------------------------------------------------------------------------
def _posres_particle(k=1.0, box=100.0):
    sp = synth.harmonic_well(dims=3, k0=k, k1=k, box=box)
    return sp


def test_baoab_harmonic_variance_is_exact():
    """BAOAB samples the exact configurational distribution of a harmonic
    oscillator at any stable step: <x^2> = kT/k, here at dt = 0.5 and
    omega = 1, where a step-size error of O(dt^2) would be ~6 %."""
    sp = _posres_particle(k=1.0)
    run = synth.harmonic_run(seed=21, n_walkers=8, dt=0.5)
    run.lambda_dynamics = False
    run.abf_on = False
    sim = oracle.Simulation(sp, run)
    acc, n = 0.0, 0
    for _ in range(3000):
        sim.run(1)
        d = sim.a["x"][:, 0, :] - sp.box / 2.0
        acc += float((d * d).sum())
        n += d.size
    assert acc / n == pytest.approx(1.0, abs=0.03)


def test_frictionless_step_is_time_reversible():
    """With gamma = 0 the B-A-(O=identity)-A-B step is time-reversible: run
    forward, negate the velocities, run again and the start comes back."""
    sp = synth.lj_fluid(cells=3)
    run = synth.lj_fluid_run(seed=5, n_walkers=1)
    run.gamma = 0.0
    run.dt = 0.002
    run.lambda_dynamics = False
    run.abf_on = False
    st = synth.initial_state(sp, run, lam0=[0.6])
    sim = oracle.Simulation(sp, run, st)
    x0 = sim.a["x"].copy()
    sim.run(300)
    assert np.abs(sim.a["x"] - x0).max() > 0.1
    sim.a["v"] *= -1.0
    sim.run(300)
    d = sim.a["x"] - x0
    d -= sp.box * np.round(d / sp.box)
    assert np.abs(d).max() < 1e-8


def test_energy_conservation_smooth_potential():
    """gamma = 0 on a smooth potential (flexible waters, bonds and angles
    only): the total energy does not drift and its fluctuation shrinks as
    dt^2 (the shadow-Hamiltonian property of velocity Verlet)."""
    sp = synth.water_box(8, 1, seed=4, box=3.0)
    sp = synth.with_changes(sp, charge=np.zeros(sp.n), epsilon=np.zeros(sp.n))
    amp = {}
    for dt in (0.0002, 0.0001):
        run = synth.water_run(seed=5, walkers_per_stage=1)
        run.stages = [synth.Stage(0.0, 1.0, 10, 1)]
        run.gamma = 0.0
        run.dt = dt
        run.lambda_dynamics = False
        run.abf_on = False
        sim = oracle.Simulation(sp, run)

        def total():
            x, v = sim.a["x"][0], sim.a["v"][0]
            return (oracle.energy_forces(sim.osys, x, 0.0)["U"]
                    + 0.5 * float((sp.mass[:, None] * v * v).sum()))

        e0 = total()
        es = []
        for _ in range(40):
            sim.run(int(round(0.01 / dt)))
            es.append(total())
        es = np.asarray(es)
        amp[dt] = np.abs(es - e0).max()
        assert amp[dt] < 3e-3 * abs(e0)
        assert abs(es[20:].mean() - es[:20].mean()) < 0.2 * amp[dt] + 1e-9
    assert 2.5 < amp[0.0002] / amp[0.0001] < 6.0


def test_reflection_keeps_lambda_in_stage():
    sp = synth.harmonic_well(dims=1)
    run = synth.harmonic_run(seed=3, n_walkers=4)
    run.stages = [synth.Stage(0.2, 0.6, 20, 4)]
    run.gamma_lambda = 0.1  # underdamped: hits the walls often
    st = synth.initial_state(sp, run, lam0=[0.2, 0.3, 0.5, 0.6])
    sim = oracle.Simulation(sp, run, st)
    lo, hi = 1.0, 0.0
    for _ in range(400):
        sim.run(10)
        lo = min(lo, sim.a["lam"].min())
        hi = max(hi, sim.a["lam"].max())
    assert lo >= 0.2 and hi <= 0.6
    assert lo < 0.22 and hi > 0.58


def test_sample_bookkeeping_and_shared_freq():
    sp = synth.harmonic_well(dims=1)
    for K in (1, 7):
        run = synth.harmonic_run(seed=9, n_walkers=3)
        run.shared_freq = K
        sim = oracle.Simulation(sp, run)
        sim.run(70)
        s, _, c = sim.stage_bins(0)
        assert c.sum() == 3 * 70  # every walker's sample lands once, 70 = 10 K'
        assert not sim.a["dl_count"].any()


def _harmonic_delta_a(seed, dims, n_steps, n_walkers=4, k1=4.0, theta=False):
    sp = synth.harmonic_well(dims=dims, k0=1.0, k1=k1)
    run = synth.harmonic_run(seed=seed, n_walkers=n_walkers)
    run.theta_stats = theta
    sim = oracle.Simulation(sp, run)
    sim.run(n_steps)
    return sim


@pytest.mark.slow
def test_harmonic_switch_free_energy_closed_form():
    """Delta A = (d kT / 2) ln(k1 / k0) within 0.05 kT, and every bin mean
    agrees with the exact bin-averaged mean force (kT/2) ln(k(hi)/k(lo)) / w."""
    vals = []
    for seed in range(3):
        sim = _harmonic_delta_a(100 + seed, 1, 100_000)
        grad, A, dA = sim.delta_a(0)
        vals.append(dA)
        edges = np.linspace(0, 1, 51)
        k = 1.0 + 3.0 * edges
        exact = 0.5 * np.log(k[1:] / k[:-1]) / 0.02
        assert np.all(np.isfinite(grad))
        assert np.median(np.abs(grad - exact)) < 0.05
    assert np.mean(vals) == pytest.approx(0.5 * np.log(4.0), abs=0.05)


@pytest.mark.slow
def test_delta_a_does_not_depend_on_the_bias_ramp():
    """The bias depends on lambda only, so it changes where the walkers go but
    not the conditional mean of dU/dlambda in a bin (Sec. 2.3): Delta A is the
    same closed form for a ramp that reaches full bias after 10 samples and
    one that needs 10^5 (about 8000 samples per bin here: the bias stays
    below a tenth of the mean force for the whole run)."""
    out = {}
    for n_full in (10.0, 1e5):
        vals = []
        for seed in range(3):
            sp = synth.harmonic_well(dims=1, k0=1.0, k1=4.0)
            run = synth.harmonic_run(seed=500 + seed, n_walkers=4, n_full=n_full)
            sim = oracle.Simulation(sp, run)
            sim.run(100_000)
            vals.append(sim.delta_a(0)[2])
        out[n_full] = np.mean(vals)
    for v in out.values():
        assert v == pytest.approx(0.5 * np.log(4.0), abs=0.05)
    assert abs(out[10.0] - out[1e5]) < 0.05


@pytest.mark.slow
def test_fixed_lambda_windows_closed_form():
    """Fixed-lambda windows (the comparison method of Sec. 4): each window's
    mean <dU/dlambda> is the closed form (d kT/2)(k1 - k0)/k(lambda_c) and the
    midpoint sum over windows is Delta A = (d kT/2) ln(k1/k0) (the midpoint
    rule's own error is below 1e-3 here)."""
    sp = synth.harmonic_well(dims=3)
    run, lam0 = synth.fixed_lambda_windows(synth.harmonic_run(seed=301), 10, 4)
    assert not run.lambda_dynamics and run.n_walkers == 40
    st = synth.initial_state(sp, run, lam0=lam0)
    sim = oracle.Simulation(sp, run, st)
    sim.run(100_000)
    assert np.allclose(sim.a["lam"], lam0)  # frozen
    grad, A, dA = sim.delta_a(0)
    lc = (np.arange(10) + 0.5) / 10
    exact = 1.5 * 3.0 / (1.0 + 3.0 * lc)
    np.testing.assert_allclose(grad, exact, rtol=0.08)
    assert dA == pytest.approx(1.5 * np.log(4.0), abs=0.05)


@pytest.mark.slow
def test_harmonic_switch_theta_gradient_closed_form():
    """d Delta A / d k1 = d kT / (2 k1) from the bin estimator with the
    covariance term."""
    got = []
    for seed in range(3):
        sim = _harmonic_delta_a(200 + seed, 1, 100_000, theta=True)
        got.append(sim.theta_gradient(0)[-1])
    assert np.mean(got) == pytest.approx(1.0 / (2 * 4.0), abs=0.02)


@pytest.mark.slow
def test_abf_flattens_lambda_histogram():
    """Under ABF the lambda distribution converges to uniform (Sec. 2.3);
    without the bias the walkers pile up where A(lambda) is low."""
    counts = {}
    for abf in (False, True):
        sp = synth.harmonic_well(dims=3, k0=1.0, k1=16.0)
        run = synth.harmonic_run(seed=77, n_walkers=4, n_bins=10)
        run.abf_on = abf
        sim = oracle.Simulation(sp, run)
        sim.run(60_000)
        counts[abf] = sim.stage_bins(0)[2].astype(float)
    r_plain = counts[False].max() / counts[False].min()
    r_abf = counts[True].max() / counts[True].min()
    assert r_plain > 5.0
    assert r_abf < 2.0


def test_masked_evaluation_matches_full():
    """The masked pass visits only pairs touching selected or alchemical
    atoms: forces on the selected atoms, dU/dlambda and the theta
    derivatives equal those of the full pass."""
    sp, x = _restrained_small(6)
    o = oracle.OracleSystem(sp)
    atoms = np.array([0, 4, 17, 30, sp.n - 2])
    for lam in (0.2, 0.7):
        full = oracle.energy_forces(o, x, lam)
        part = oracle.energy_forces_masked(o, x, lam, atoms)
        np.testing.assert_allclose(part["F"][atoms], full["F"][atoms], rtol=1e-12, atol=1e-10)
        assert part["dUdl"] == pytest.approx(full["dUdl"], rel=1e-12, abs=1e-12)
        np.testing.assert_allclose(part["dth"], full["dth"], rtol=1e-12, atol=1e-12)


def test_lambda_dependent_restraint_endpoints():
    """d_min(lambda) = delta/2 (1 - cos 2 pi lambda): no restraint at lambda = 0
    and 1, full distance delta at lambda = 1/2 (Sec. 4.2)."""
    r, delta, k = 0.3, 1.0, 500.0
    sp = _two_atoms(r, sig=(0, 0), eps=(0, 0), rc=2.5)
    sp = synth.with_changes(sp, lr_ij=np.array([[0, 1]], np.int32), lr_delta=delta, lr_k=k)
    o = oracle.OracleSystem(sp)
    x = sp.x.astype(np.float64)
    ra = float(x[1, 0] - x[0, 0])
    assert oracle.energy_forces(o, x, 0.0)["terms"][6] == 0.0
    assert oracle.energy_forces(o, x, 1.0)["terms"][6] == pytest.approx(0.0, abs=1e-20)
    mid = oracle.energy_forces(o, x, 0.5)
    assert mid["terms"][6] == pytest.approx(0.5 * k * (ra - delta) ** 2, rel=1e-12)
    assert mid["dUdl"] == pytest.approx(0.0, abs=1e-9)  # d_min is stationary at 1/2
    q = oracle.energy_forces(o, x, 0.25)  # d_min = delta/2, slope delta pi
    assert q["dl"][2] == pytest.approx(-k * (ra - 0.5 * delta) * delta * np.pi, rel=1e-12)


def test_pair_set_rows_is_the_pair_set_restricted_to_the_rows():
    """or_pair_set_rows returns exactly the pairs of the brute-force set
    (and of or_pair_set) touching a selected atom, in the same order."""
    sp, x = _small_water(5)
    x = x.astype(np.float32)
    o = oracle.OracleSystem(sp)
    full, fkind = oracle.pair_set(o, x, 1.0)
    brute = _brute_pairs(sp, x, 1.0)
    rng = np.random.default_rng(3)
    for k in (1, 7, sp.n // 2, sp.n):
        rows = np.sort(rng.choice(sp.n, k, replace=False))
        sel = np.zeros(sp.n, bool)
        sel[rows] = True
        got, kind = oracle.pair_set_rows(o, x, 1.0, rows)
        keep = sel[full[:, 0]] | sel[full[:, 1]]
        assert np.array_equal(got, full[keep]) and np.array_equal(kind, fkind[keep])
        assert set(map(tuple, got.tolist())) == {p for p in brute if sel[p[0]] or sel[p[1]]}
