"""Seeded synthetic systems shaped like the paper's workloads.

This module only builds inputs: positions on lattices with seeded jitter,
force-field parameters drawn from stated distributions, topologies
(bonds, angles, exclusions, restraints), Maxwell-Boltzmann initial
velocities and the run parameters of each workload.  It contains none of
the method's arithmetic (no lambda path, no potential, no integrator, no
ABF), so both the CUDA engine and the FP64 oracle consume it unchanged.

Units: the LJ-fluid workload uses reduced units (epsilon = sigma = m = kT = 1);
the water workloads use nm, ps, amu, kJ/mol and elementary charges.

The paper's own systems (AMOEBA/CHARMM ions, CB8, lysozyme, CypD) need force
fields and structures that are not available; these stand-ins reproduce
the shapes: a plain LJ fluid with one alchemical solute, flexible 3-site
water boxes with a small neutral alchemical solute, uneven batches of such
boxes, and a large restrained complex.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Tuple

import numpy as np

KB_KJ_PER_MOL_K = 0.0083144626
COULOMB_KJ_NM = 138.935458  # kJ mol^-1 nm e^-2
TEMPERATURE_K = 300.0
# m_lambda = 150000 kcal/mol fs^2 expressed in kJ/mol ps^2 (Sec. 2.2)
M_LAMBDA_KJ_PS2 = 150000.0 * 4.184 * 1.0e-6
GAMMA_LAMBDA_PS = 1000.0

# 3-site flexible water (TIP3P-like charges and O-O Lennard-Jones)
WATER_Q_O, WATER_Q_H = -0.834, 0.417
WATER_SIG_O, WATER_EPS_O = 0.315, 0.636
WATER_R_OH, WATER_THETA_DEG = 0.09572, 104.52
WATER_KB, WATER_KTHETA = 502416.0, 628.02
MASS_O, MASS_H, MASS_C = 15.9994, 1.008, 12.011
CHAIN_R0, CHAIN_KB = 0.15, 2.5e5


@dataclass
class SystemSpec:
    name: str
    box: float
    mass: np.ndarray
    charge: np.ndarray
    sigma: np.ndarray
    epsilon: np.ndarray
    alch: np.ndarray
    excl_group: np.ndarray
    excl_extra: np.ndarray
    x: np.ndarray  # (n, 3) float32 initial configuration
    bond_ij: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    bond_r0: np.ndarray = field(default_factory=lambda: np.zeros(0))
    bond_k: np.ndarray = field(default_factory=lambda: np.zeros(0))
    angle_ijk: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), np.int32))
    angle_t0: np.ndarray = field(default_factory=lambda: np.zeros(0))
    angle_k: np.ndarray = field(default_factory=lambda: np.zeros(0))
    posres_idx: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    posres_x0: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    posres_k: float = 0.0
    fb_a: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    fb_b: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    fb_d0: float = 0.0
    fb_k: float = 0.0
    lh_idx: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    lh_x0: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    lh_k0: float = 0.0
    lh_k1: float = 0.0
    lh_dims: int = 3
    # lambda-dependent distance restraint: atom pairs kept at least
    # delta/2 (1 - cos 2 pi lambda) apart with force constant lr_k
    lr_ij: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    lr_delta: float = 0.0
    lr_k: float = 0.0
    r_cut: float = 1.0
    eps_rf: float = 78.0
    coul: float = COULOMB_KJ_NM
    b_v: float = 0.5
    b_e: float = 0.5
    sc_alpha: float = 0.5
    sc_n: int = 1
    sc_m: int = 1

    @property
    def n(self) -> int:
        return int(self.mass.shape[0])

    @property
    def n_alch(self) -> int:
        return int(self.alch.sum())


@dataclass
class Stage:
    lo: float
    hi: float
    n_bins: int
    n_walkers: int


@dataclass
class RunSpec:
    kT: float
    dt: float
    gamma: float
    m_lambda: float
    gamma_lambda: float
    skin: float
    n_full: float
    shared_freq: int
    seed: int
    stages: List[Stage]
    lambda_dynamics: bool = True
    abf_on: bool = True
    theta_stats: bool = False

    @property
    def n_walkers(self) -> int:
        return sum(s.n_walkers for s in self.stages)

    def walker_stage(self) -> np.ndarray:
        out = []
        for k, s in enumerate(self.stages):
            out += [k] * s.n_walkers
        return np.asarray(out, np.int32)


@dataclass
class WalkerState:
    x: np.ndarray     # (W, n, 3) float32
    v: np.ndarray     # (W, n, 3) float32
    lam: np.ndarray   # (W,) float64
    plam: np.ndarray  # (W,) float64


def _empty_excl(n: int) -> np.ndarray:
    return np.full((n, 4), -1, np.int32)


# --------------------------------------------------------------------------
# Workload 1: LJ fluid with one alchemical LJ solute (reduced units)
# --------------------------------------------------------------------------
def lj_fluid(seed: int = 8006, cells: int = 4, density: float = 0.8, jitter: float = 0.05,
             r_cut: float = 2.5) -> SystemSpec:
    """256 LJ atoms (eps = sigma = 1) on an FCC lattice at the given density,
    with uniform jitter of +-jitter sigma, plus one alchemical solute
    (eps = 1.5, sigma = 1.2) at the octahedral hole (a/2, a/2, a/2)."""
    rng = np.random.default_rng(seed)
    n_lat = 4 * cells ** 3
    box = (n_lat / density) ** (1.0 / 3.0)
    a = box / cells
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    pts = []
    for i in range(cells):
        for j in range(cells):
            for k in range(cells):
                for b in basis:
                    pts.append((np.array([i, j, k]) + b) * a)
    pts = np.asarray(pts)
    pts += rng.uniform(-jitter, jitter, pts.shape)
    solute = np.array([[a / 2, a / 2, a / 2]])
    x = np.concatenate([pts, solute]) % box
    n = x.shape[0]
    sigma = np.ones(n)
    eps = np.ones(n)
    sigma[-1], eps[-1] = 1.2, 1.5
    alch = np.zeros(n, np.uint8)
    alch[-1] = 1
    return SystemSpec(name="lj_fluid_256", box=box, mass=np.ones(n), charge=np.zeros(n),
                      sigma=sigma, epsilon=eps, alch=alch, excl_group=np.full(n, -1, np.int32),
                      excl_extra=_empty_excl(n), x=x.astype(np.float32), r_cut=r_cut,
                      eps_rf=0.0, coul=0.0, b_v=1.0, b_e=0.0, sc_alpha=0.5)


def lj_fluid_run(seed: int = 8006, n_walkers: int = 4, n_bins: int = 50) -> RunSpec:
    return RunSpec(kT=1.0, dt=0.005, gamma=1.0, m_lambda=20.0, gamma_lambda=1.0, skin=0.3,
                   n_full=100.0, shared_freq=1, seed=seed,
                   stages=[Stage(0.0, 1.0, n_bins, n_walkers)])


# --------------------------------------------------------------------------
# Water boxes with a neutral alchemical chain solute (nm, ps, kJ/mol)
# --------------------------------------------------------------------------
def _water_molecule(origin: np.ndarray) -> np.ndarray:
    half = np.deg2rad(WATER_THETA_DEG) / 2.0
    h1 = origin + WATER_R_OH * np.array([np.sin(half), np.cos(half), 0.0])
    h2 = origin + WATER_R_OH * np.array([-np.sin(half), np.cos(half), 0.0])
    return np.stack([origin, h1, h2])


def _solute_params(rng, n_sol: int):
    q = rng.normal(0.0, 0.3, n_sol)
    if n_sol > 0:
        q -= q.mean()
    sig = rng.uniform(0.3, 0.4, n_sol)
    eps = rng.uniform(0.2, 0.6, n_sol)
    return q, sig, eps


def water_box(n_waters: int = 4096, n_solute: int = 12, seed: int = 8007, box: float | None = None,
              r_cut: float = 1.0, eps_rf: float = 78.0, name: str | None = None) -> SystemSpec:
    """n_waters flexible 3-site waters on a cubic grid (one common
    orientation), plus an n_solute-site neutral alchemical chain (0.15 nm
    harmonic bonds) along x at the box centre.  The box edge defaults to the
    4096-water / 5 nm density."""
    rng = np.random.default_rng(seed)
    if box is None:
        box = (n_waters / 32.768) ** (1.0 / 3.0)
    per_side = int(np.ceil(n_waters ** (1.0 / 3.0) - 1e-9))
    spacing = box / per_side
    sites = []
    for i in range(per_side):
        for j in range(per_side):
            for k in range(per_side):
                sites.append((i + 0.25, j + 0.25, k + 0.25))
    sites = np.asarray(sites[:n_waters]) * spacing
    xw = np.concatenate([_water_molecule(o) for o in sites])
    nw = 3 * n_waters
    # the chain runs along x through the channel between four water rows
    centre = np.array([box / 2.0, (per_side // 2 - 0.25) * spacing, (per_side // 2 - 0.25) * spacing])
    xs = np.zeros((n_solute, 3))
    xs[:, 0] = (np.arange(n_solute) - (n_solute - 1) / 2.0) * CHAIN_R0
    xs += centre
    x = np.concatenate([xw, xs]) % box
    n = nw + n_solute
    mass = np.empty(n)
    charge = np.empty(n)
    sigma = np.zeros(n)
    eps = np.zeros(n)
    mass[0:nw:3], mass[1:nw:3], mass[2:nw:3] = MASS_O, MASS_H, MASS_H
    charge[0:nw:3], charge[1:nw:3], charge[2:nw:3] = WATER_Q_O, WATER_Q_H, WATER_Q_H
    sigma[0:nw:3], eps[0:nw:3] = WATER_SIG_O, WATER_EPS_O
    q, sg, ep = _solute_params(rng, n_solute)
    mass[nw:], charge[nw:], sigma[nw:], eps[nw:] = MASS_C, q, sg, ep
    alch = np.zeros(n, np.uint8)
    alch[nw:] = 1
    group = np.empty(n, np.int32)
    group[:nw] = np.repeat(np.arange(n_waters), 3)
    group[nw:] = n_waters
    o = np.arange(n_waters) * 3
    bonds = np.concatenate([np.stack([o, o + 1], 1), np.stack([o, o + 2], 1)])
    b_r0 = np.full(2 * n_waters, WATER_R_OH)
    b_k = np.full(2 * n_waters, WATER_KB)
    if n_solute > 1:
        s = nw + np.arange(n_solute - 1)
        bonds = np.concatenate([bonds, np.stack([s, s + 1], 1)])
        b_r0 = np.concatenate([b_r0, np.full(n_solute - 1, CHAIN_R0)])
        b_k = np.concatenate([b_k, np.full(n_solute - 1, CHAIN_KB)])
    angles = np.stack([o + 1, o, o + 2], 1)
    return SystemSpec(
        name=name or f"water{n_waters}_solute{n_solute}", box=float(box), mass=mass,
        charge=charge, sigma=sigma, epsilon=eps, alch=alch, excl_group=group,
        excl_extra=_empty_excl(n), x=x.astype(np.float32), bond_ij=bonds.astype(np.int32),
        bond_r0=b_r0, bond_k=b_k, angle_ijk=angles.astype(np.int32),
        angle_t0=np.full(n_waters, np.deg2rad(WATER_THETA_DEG)),
        angle_k=np.full(n_waters, WATER_KTHETA), r_cut=r_cut, eps_rf=eps_rf,
        coul=COULOMB_KJ_NM, b_v=0.5, b_e=0.5, sc_alpha=0.5)


def water_run(seed: int = 8007, walkers_per_stage: int = 8, n_bins: int = 100,
              n_full: float = 200.0, skin: float = 0.1) -> RunSpec:
    """Two stages (vdW on [0, 0.5], Coulomb on [0.5, 1]); 1 fs steps at 300 K;
    gamma = 1 ps^-1 for atoms; m_lambda and gamma_lambda from Sec. 2.2."""
    kT = KB_KJ_PER_MOL_K * TEMPERATURE_K
    return RunSpec(kT=kT, dt=0.001, gamma=1.0, m_lambda=M_LAMBDA_KJ_PS2,
                   gamma_lambda=GAMMA_LAMBDA_PS, skin=skin, n_full=n_full, shared_freq=1,
                   seed=seed, stages=[Stage(0.0, 0.5, n_bins, walkers_per_stage),
                                      Stage(0.5, 1.0, n_bins, walkers_per_stage)])


# the uneven batch: water counts and solute sizes per system
UNEVEN_WATERS = (256, 512, 1024, 2048, 3072, 4096, 6144, 8192)
UNEVEN_SOLUTES = (4, 9, 14, 19, 25, 30, 35, 40)


def uneven_batch(seed: int = 8008) -> List[SystemSpec]:
    """Eight water boxes at the 4096-water density; the 256-water box
    (edge 1.98 nm) takes r_c = 0.85 nm so that it stays above twice the
    list radius."""
    out = []
    for k, (nw, ns) in enumerate(zip(UNEVEN_WATERS, UNEVEN_SOLUTES)):
        rc = 0.85 if nw == 256 else 1.0
        out.append(water_box(nw, ns, seed=seed + 100 * k, r_cut=rc))
    return out


def uneven_run(seed: int = 8008, walkers_per_system: int = 8) -> RunSpec:
    r = water_run(seed=seed, walkers_per_stage=walkers_per_system // 2)
    return r


# --------------------------------------------------------------------------
# Workload 5: large restrained complex
# --------------------------------------------------------------------------
def _serpentine(n_sites: int, lattice: float, dims: Tuple[int, int, int]) -> np.ndarray:
    """A boustrophedon path on a cubic lattice, with one extra site at the
    midpoint of every lattice step, truncated to n_sites points."""
    nx, ny, nz = dims
    pts = []
    for k in range(nz):
        ys = range(ny) if k % 2 == 0 else range(ny - 1, -1, -1)
        for jj, j in enumerate(ys):
            xs = range(nx) if (jj + k * ny) % 2 == 0 else range(nx - 1, -1, -1)
            for i in xs:
                pts.append((i, j, k))
    pts = np.asarray(pts, float) * lattice
    out = [pts[0]]
    for p, q in zip(pts[:-1], pts[1:]):
        out.append(0.5 * (p + q))
        out.append(q)
        if len(out) >= n_sites:
            break
    return np.asarray(out[:n_sites])


def large_complex(seed: int = 8010, n_waters: int = 31000, n_chain: int = 3000,
                  n_lig: int = 40, r_cut: float = 1.2, density_atoms: float = 98.4,
                  jitter: float = 0.005) -> SystemSpec:
    """31000 flexible waters, a 3000-site bonded chain held by positional
    restraints, and a 40-site alchemical ligand with a flat-bottom restraint
    between its centre of mass and that of the chain sites near it.  The box
    is sized to liquid-water atom density (the 8.2 nm edge would overlap
    atoms)."""
    rng = np.random.default_rng(seed)
    n_atoms = 3 * n_waters + n_chain + n_lig
    box = (n_atoms / density_atoms) ** (1.0 / 3.0)
    lat = 0.3
    chain = _serpentine(n_chain, lat, (12, 12, 11))
    chain += np.array([box / 2 - 1.65, box / 2 - 1.65, box / 2 - 1.5])
    lig = _serpentine(n_lig, lat, (4, 3, 2))
    lig += np.array([box / 2 - 0.45, box / 2 - 0.3, box / 2 + 1.95])
    solid = np.concatenate([chain, lig])
    # water grid: finest cubic grid whose free sites cover n_waters
    from scipy.spatial import cKDTree

    tree = cKDTree(solid % box, boxsize=box)
    per_side = int(np.ceil((n_waters * 1.15) ** (1.0 / 3.0)))
    while True:
        spacing = box / per_side
        g = (np.stack(np.meshgrid(*[np.arange(per_side)] * 3, indexing="ij"), -1)
             .reshape(-1, 3) + 0.25) * spacing
        # drop grid sites within 0.33 nm of a chain or ligand site (periodic)
        dist, _ = tree.query(g % box, k=1, distance_upper_bound=0.33)
        free = g[~np.isfinite(dist)]
        if len(free) >= n_waters:
            break
        per_side += 1
    pick = np.sort(rng.choice(len(free), n_waters, replace=False))
    sites = free[pick]
    xw = np.concatenate([_water_molecule(o) for o in sites])
    nw = 3 * n_waters
    x = np.concatenate([xw, chain, lig])
    # seeded jitter: lattice starts put many pair distances exactly on the
    # cutoff (1.2 nm = 8 x 0.15 nm), where any rounding flips the pair
    x = (x + rng.uniform(-jitter, jitter, x.shape)) % box
    n = x.shape[0]
    mass = np.empty(n)
    charge = np.empty(n)
    sigma = np.zeros(n)
    eps = np.zeros(n)
    mass[0:nw:3], mass[1:nw:3], mass[2:nw:3] = MASS_O, MASS_H, MASS_H
    charge[0:nw:3], charge[1:nw:3], charge[2:nw:3] = WATER_Q_O, WATER_Q_H, WATER_Q_H
    sigma[0:nw:3], eps[0:nw:3] = WATER_SIG_O, WATER_EPS_O
    qc, sc, ec = _solute_params(rng, n_chain)
    ql, sl, el = _solute_params(rng, n_lig)
    c0, l0 = nw, nw + n_chain
    mass[c0:] = MASS_C
    charge[c0:l0], sigma[c0:l0], eps[c0:l0] = qc, sc, ec
    charge[l0:], sigma[l0:], eps[l0:] = ql, sl, el
    alch = np.zeros(n, np.uint8)
    alch[l0:] = 1
    group = np.full(n, -1, np.int32)
    group[:nw] = np.repeat(np.arange(n_waters), 3)
    group[l0:] = n_waters
    extra = _empty_excl(n)
    for i in range(n_chain):  # chain 1-2 and 1-3 exclusions
        partners = [j for j in (i - 2, i - 1, i + 1, i + 2) if 0 <= j < n_chain]
        extra[c0 + i, :len(partners)] = c0 + np.asarray(partners)
    o = np.arange(n_waters) * 3
    sb = c0 + np.arange(n_chain - 1)
    lb = l0 + np.arange(n_lig - 1)
    bonds = np.concatenate([np.stack([o, o + 1], 1), np.stack([o, o + 2], 1),
                            np.stack([sb, sb + 1], 1), np.stack([lb, lb + 1], 1)])
    b_r0 = np.concatenate([np.full(2 * n_waters, WATER_R_OH), np.full(n_chain - 1, CHAIN_R0),
                           np.full(n_lig - 1, CHAIN_R0)])
    b_k = np.concatenate([np.full(2 * n_waters, WATER_KB), np.full(n_chain - 1, CHAIN_KB),
                          np.full(n_lig - 1, CHAIN_KB)])
    angles = np.stack([o + 1, o, o + 2], 1)
    lig_com = lig.mean(0)
    d = chain - lig_com
    near_chain = np.nonzero((d * d).sum(1) < 1.2 ** 2)[0]
    if near_chain.size == 0:
        near_chain = np.argsort((d * d).sum(1))[:16]
    return SystemSpec(
        name="complex96k", box=float(box), mass=mass, charge=charge, sigma=sigma, epsilon=eps,
        alch=alch, excl_group=group, excl_extra=extra, x=x.astype(np.float32),
        bond_ij=bonds.astype(np.int32), bond_r0=b_r0, bond_k=b_k,
        angle_ijk=angles.astype(np.int32),
        angle_t0=np.full(n_waters, np.deg2rad(WATER_THETA_DEG)),
        angle_k=np.full(n_waters, WATER_KTHETA),
        posres_idx=(c0 + np.arange(n_chain)).astype(np.int32),
        posres_x0=x[c0:l0].astype(np.float64), posres_k=1000.0,
        fb_a=(l0 + np.arange(n_lig)).astype(np.int32),
        fb_b=(c0 + near_chain).astype(np.int32), fb_d0=1.0, fb_k=1000.0,
        r_cut=r_cut, eps_rf=78.0, coul=COULOMB_KJ_NM, b_v=0.5, b_e=0.5, sc_alpha=0.5)


def large_complex_run(seed: int = 8010, walkers_per_stage: int = 8) -> RunSpec:
    return water_run(seed=seed, walkers_per_stage=walkers_per_stage)


# --------------------------------------------------------------------------
# Analytic test: a lambda-switched harmonic well
# --------------------------------------------------------------------------
def harmonic_well(dims: int = 1, k0: float = 1.0, k1: float = 4.0, box: float = 100.0) -> SystemSpec:
    """One free particle (m = 1) in a well 1/2 ((1-lam) k0 + lam k1) |x|^2
    over `dims` Cartesian components, centred in a large box."""
    n = 1
    x = np.full((1, 3), box / 2.0, np.float32)
    return SystemSpec(
        name=f"harmonic{dims}d", box=box, mass=np.ones(n), charge=np.zeros(n),
        sigma=np.zeros(n), epsilon=np.zeros(n), alch=np.zeros(n, np.uint8),
        excl_group=np.full(n, -1, np.int32), excl_extra=_empty_excl(n), x=x,
        lh_idx=np.zeros(1, np.int32), lh_x0=x.astype(np.float64), lh_k0=k0, lh_k1=k1,
        lh_dims=dims, r_cut=2.0, eps_rf=0.0, coul=0.0, b_v=1.0, b_e=0.0)


def harmonic_run(seed: int = 8011, n_walkers: int = 4, n_bins: int = 50, dt: float = 0.005,
                 n_full: float = 100.0) -> RunSpec:
    return RunSpec(kT=1.0, dt=dt, gamma=1.0, m_lambda=20.0, gamma_lambda=1.0, skin=0.3,
                   n_full=n_full, shared_freq=1, seed=seed,
                   stages=[Stage(0.0, 1.0, n_bins, n_walkers)])


# --------------------------------------------------------------------------
# Fixed-lambda windows (the comparison method of Sec. 4: thermodynamic
# integration over frozen lambda values)
# --------------------------------------------------------------------------
def fixed_lambda_windows(run: RunSpec, windows_per_stage: int, walkers_per_window: int = 1):
    """The same stages cut into `windows_per_stage` windows each, one bin per
    window and `walkers_per_window` walkers frozen at each window centre
    (lambda dynamics and the bias off).  The midpoint-rule sum of the bin
    means is then the TI estimate over the windows.  Returns (run, lam0)."""
    stages, lam0 = [], []
    for st in run.stages:
        w = (st.hi - st.lo) / windows_per_stage
        stages.append(Stage(st.lo, st.hi, windows_per_stage, windows_per_stage * walkers_per_window))
        for k in range(windows_per_stage):
            lam0 += [st.lo + (k + 0.5) * w] * walkers_per_window
    out = RunSpec(kT=run.kT, dt=run.dt, gamma=run.gamma, m_lambda=run.m_lambda,
                  gamma_lambda=run.gamma_lambda, skin=run.skin, n_full=run.n_full,
                  shared_freq=run.shared_freq, seed=run.seed, stages=stages,
                  lambda_dynamics=False, abf_on=False, theta_stats=run.theta_stats)
    return out, lam0


# --------------------------------------------------------------------------
# Initial walker states
# --------------------------------------------------------------------------
def initial_state(spec: SystemSpec, run: RunSpec, seed: int | None = None,
                  lam0: List[float] | None = None) -> WalkerState:
    """Every walker starts from the system's configuration with its own
    Maxwell-Boltzmann velocities; lambda starts at its stage's lower wall
    (or lam0) with a Maxwell-Boltzmann momentum."""
    rng = np.random.default_rng(run.seed if seed is None else seed)
    W, n = run.n_walkers, spec.n
    x = np.broadcast_to(spec.x, (W, n, 3)).astype(np.float32).copy()
    with np.errstate(divide="ignore"):  # a massless atom is refused by the engine
        sd = np.sqrt(run.kT / spec.mass)[None, :, None]
    v = (rng.standard_normal((W, n, 3)) * sd).astype(np.float32)
    stages = run.walker_stage()
    if lam0 is None:
        lam = np.asarray([run.stages[s].lo for s in stages], np.float64)
    else:
        lam = np.asarray(lam0, np.float64)
    plam = rng.standard_normal(W) * np.sqrt(run.m_lambda * run.kT)
    return WalkerState(x=x, v=v, lam=lam, plam=plam)


def with_changes(spec: SystemSpec, **kw) -> SystemSpec:
    return replace(spec, **kw)
