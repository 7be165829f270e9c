"""FP64 CPU oracle for the lambda-ABF multiple-walker step (arXiv 2307.08006).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA engine in ``paper_2307_08006_gb300``) never imports, links or
executes anything here, and this package imports nothing from the engine
except the seeded input generators in ``paper_2307_08006_gb300.synth``,
which hold none of the method's arithmetic.

The C source (``labf_oracle.c``) is the oracle proper; this module compiles
it with gcc (``-O2 -ffp-contract=off -fopenmp``) and exposes it through
ctypes with numpy arrays.  See the C file's header for the paper passages
each function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "labf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblabf_oracle.so")
_lock = threading.Lock()
_lib = None

N_TERMS = 7
TERM_NAMES = ("lj", "rf", "sc_lj", "sc_rf", "bond", "angle", "restraint")


def build(force: bool = False) -> str:
    """Compile the oracle shared library (a few seconds with gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    deps = [_SRC, os.path.join(_HERE, "labf_oracle.h")]
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(d) for d in deps)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB_PATH)
            _declare(lib)
            _lib = lib
    return _lib


class _System(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("box", C.c_double),
        ("mass", C.c_void_p), ("charge", C.c_void_p), ("sigma", C.c_void_p),
        ("epsilon", C.c_void_p), ("alch", C.c_void_p), ("excl_group", C.c_void_p),
        ("excl_extra", C.c_void_p),
        ("n_bonds", C.c_int), ("bond_ij", C.c_void_p), ("bond_r0", C.c_void_p),
        ("bond_k", C.c_void_p),
        ("n_angles", C.c_int), ("angle_ijk", C.c_void_p), ("angle_t0", C.c_void_p),
        ("angle_k", C.c_void_p),
        ("n_posres", C.c_int), ("posres_idx", C.c_void_p), ("posres_x0", C.c_void_p),
        ("posres_k", C.c_double),
        ("n_fb_a", C.c_int), ("fb_a", C.c_void_p), ("n_fb_b", C.c_int), ("fb_b", C.c_void_p),
        ("fb_d0", C.c_double), ("fb_k", C.c_double),
        ("n_lh", C.c_int), ("lh_idx", C.c_void_p), ("lh_x0", C.c_void_p),
        ("lh_k0", C.c_double), ("lh_k1", C.c_double), ("lh_dims", C.c_int),
        ("n_lr", C.c_int), ("lr_ij", C.c_void_p), ("lr_delta", C.c_double), ("lr_k", C.c_double),
        ("r_cut", C.c_double), ("eps_rf", C.c_double), ("coul", C.c_double),
        ("b_v", C.c_double), ("b_e", C.c_double),
        ("sc_alpha", C.c_double), ("sc_n", C.c_int), ("sc_m", C.c_int),
    ]


class _Run(C.Structure):
    _fields_ = [
        ("kT", C.c_double), ("dt", C.c_double), ("gamma", C.c_double),
        ("m_lambda", C.c_double), ("gamma_lambda", C.c_double),
        ("lambda_dynamics", C.c_int), ("abf_on", C.c_int), ("n_full", C.c_double),
        ("shared_freq", C.c_int), ("seed", C.c_uint32), ("n_stages", C.c_int),
        ("stage_lo", C.c_void_p), ("stage_hi", C.c_void_p), ("stage_bins", C.c_void_p),
        ("theta_stats", C.c_int),
    ]


class _State(C.Structure):
    _fields_ = [
        ("n_walkers", C.c_int), ("walker_stage", C.c_void_p),
        ("x", C.c_void_p), ("v", C.c_void_p), ("lam", C.c_void_p), ("plam", C.c_void_p),
        ("step", C.c_void_p), ("F", C.c_void_p), ("G", C.c_void_p), ("s", C.c_void_p),
        ("dth", C.c_void_p), ("d2th", C.c_void_p),
        ("abf_sum", C.c_void_p), ("abf_sumsq", C.c_void_p), ("abf_count", C.c_void_p),
        ("dl_sum", C.c_void_p), ("dl_sumsq", C.c_void_p), ("dl_count", C.c_void_p),
        ("th_d2", C.c_void_p), ("th_d", C.c_void_p), ("th_sd", C.c_void_p),
    ]


def _declare(lib):
    P = C.c_void_p
    lib.or_n_theta.argtypes = [C.POINTER(_System)]
    lib.or_n_theta.restype = C.c_int
    lib.or_lambda_path.argtypes = [C.c_double, C.c_double, C.c_double, P]
    lib.or_philox4x32_10.argtypes = [P, P, P]
    lib.or_normals4.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint32, P]
    lib.or_quantize.argtypes = [C.c_int, P, C.c_double, P]
    lib.or_list_threshold.argtypes = [C.c_double, C.c_double]
    lib.or_list_threshold.restype = C.c_int64
    lib.or_pair_set.argtypes = [C.POINTER(_System), P, C.c_double, C.c_int64, P, P, C.c_int64]
    lib.or_pair_set.restype = C.c_int64
    lib.or_pair_set_rows.argtypes = [C.POINTER(_System), P, C.c_double, C.c_int64, P, P, P, C.c_int64]
    lib.or_pair_set_rows.restype = C.c_int64
    lib.or_energy_forces.argtypes = [C.POINTER(_System), P, C.c_double, P, P, P, P, P, P]
    lib.or_energy_forces_masked.argtypes = [C.POINTER(_System), P, C.c_double, P, P, P, P, P, P, P]
    lib.or_set_threads.argtypes = [C.c_int]
    lib.or_get_max_threads.restype = C.c_int
    lib.or_bin.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int]
    lib.or_bin.restype = C.c_int
    lib.or_prime.argtypes = [C.POINTER(_System), C.POINTER(_Run), C.POINTER(_State)]
    lib.or_run.argtypes = [C.POINTER(_System), C.POINTER(_Run), C.POINTER(_State), C.c_int]
    lib.or_ti.argtypes = [P, P, C.c_int, C.c_double, C.c_double, P, P, P]
    lib.or_theta_gradient.argtypes = [P, P, P, P, P, C.c_int, C.c_double, C.c_double, C.c_int,
                                      C.c_double, P]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OracleSystem:
    """A system description in the layout the C oracle reads; keeps its
    arrays alive for the lifetime of the object."""

    def __init__(self, spec):
        # the soft-core derivative carries n lambda_v^(n-1) and
        # m (1 - lambda_v)^(m-1): integer powers below 1 are not in the
        # method's family (Beutler form, n, m >= 1) and give 0 * inf at the ends
        if int(spec.sc_n) < 1 or int(spec.sc_m) < 1:
            raise ValueError(f"soft-core powers must be >= 1 (sc_n={spec.sc_n}, sc_m={spec.sc_m})")
        self.spec = spec
        keep = {}

        def arr(name, a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep[name] = a
            return _ptr(a)

        s = _System()
        s.n = spec.n
        s.box = float(spec.box)
        s.mass = arr("mass", spec.mass, np.float64)
        s.charge = arr("charge", spec.charge, np.float64)
        s.sigma = arr("sigma", spec.sigma, np.float64)
        s.epsilon = arr("epsilon", spec.epsilon, np.float64)
        s.alch = arr("alch", spec.alch, np.uint8)
        s.excl_group = arr("excl_group", spec.excl_group, np.int32)
        s.excl_extra = arr("excl_extra", spec.excl_extra, np.int32)
        s.n_bonds = len(spec.bond_r0)
        s.bond_ij = arr("bond_ij", spec.bond_ij.reshape(-1, 2), np.int32)
        s.bond_r0 = arr("bond_r0", spec.bond_r0, np.float64)
        s.bond_k = arr("bond_k", spec.bond_k, np.float64)
        s.n_angles = len(spec.angle_t0)
        s.angle_ijk = arr("angle_ijk", spec.angle_ijk.reshape(-1, 3), np.int32)
        s.angle_t0 = arr("angle_t0", spec.angle_t0, np.float64)
        s.angle_k = arr("angle_k", spec.angle_k, np.float64)
        s.n_posres = len(spec.posres_idx)
        s.posres_idx = arr("posres_idx", spec.posres_idx, np.int32)
        s.posres_x0 = arr("posres_x0", spec.posres_x0.reshape(-1, 3), np.float64)
        s.posres_k = float(spec.posres_k)
        s.n_fb_a = len(spec.fb_a)
        s.fb_a = arr("fb_a", spec.fb_a, np.int32)
        s.n_fb_b = len(spec.fb_b)
        s.fb_b = arr("fb_b", spec.fb_b, np.int32)
        s.fb_d0, s.fb_k = float(spec.fb_d0), float(spec.fb_k)
        s.n_lh = len(spec.lh_idx)
        s.lh_idx = arr("lh_idx", spec.lh_idx, np.int32)
        s.lh_x0 = arr("lh_x0", spec.lh_x0.reshape(-1, 3), np.float64)
        s.lh_k0, s.lh_k1, s.lh_dims = float(spec.lh_k0), float(spec.lh_k1), int(spec.lh_dims)
        s.n_lr = len(spec.lr_ij)
        s.lr_ij = arr("lr_ij", np.asarray(spec.lr_ij).reshape(-1, 2), np.int32)
        s.lr_delta, s.lr_k = float(spec.lr_delta), float(spec.lr_k)
        s.r_cut, s.eps_rf, s.coul = float(spec.r_cut), float(spec.eps_rf), float(spec.coul)
        s.b_v, s.b_e = float(spec.b_v), float(spec.b_e)
        s.sc_alpha, s.sc_n, s.sc_m = float(spec.sc_alpha), int(spec.sc_n), int(spec.sc_m)
        self._keep = keep
        self.c = s
        self.n_theta = _load().or_n_theta(C.byref(s))


def lambda_path(lam: float, b_v: float, b_e: float) -> np.ndarray:
    out = np.zeros(4)
    _load().or_lambda_path(float(lam), float(b_v), float(b_e), _ptr(out))
    return out


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _load().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def normals4(seed: int, walker: int, step: int, idx: int, tag: int) -> np.ndarray:
    z = np.zeros(4)
    _load().or_normals4(seed, walker, step, idx, tag, _ptr(z))
    return z


def quantize(x: np.ndarray, box_inv: float) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    u = np.zeros(x.shape, np.uint32)
    _load().or_quantize(x.size // 3, _ptr(x), float(box_inv), _ptr(u))
    return u


def list_threshold(r_list: float, box_inv: float) -> int:
    return int(_load().or_list_threshold(float(r_list), float(box_inv)))


def pair_set(osys: OracleSystem, x: np.ndarray, r_list: float):
    """(pairs (M, 2) int32 with i < j, kind (M,) 0 = normal, 1 = alchemical)."""
    x = np.ascontiguousarray(x, np.float32)
    box_inv = 1.0 / osys.spec.box
    R = list_threshold(r_list, box_inv)
    lib = _load()
    cnt = lib.or_pair_set(C.byref(osys.c), _ptr(x), box_inv, R, None, None, 0)
    pairs = np.zeros((max(cnt, 1), 2), np.int32)
    kind = np.zeros(max(cnt, 1), np.uint8)
    lib.or_pair_set(C.byref(osys.c), _ptr(x), box_inv, R, _ptr(pairs), _ptr(kind), cnt)
    return pairs[:cnt], kind[:cnt]


def pair_set_rows(osys: OracleSystem, x: np.ndarray, r_list: float, atoms):
    """The pairs of pair_set that involve at least one of `atoms` (same
    definition and order), for checking very large systems on a sample."""
    x = np.ascontiguousarray(x, np.float32)
    box_inv = 1.0 / osys.spec.box
    R = list_threshold(r_list, box_inv)
    rows = np.zeros(osys.spec.n, np.uint8)
    rows[np.asarray(atoms)] = 1
    lib = _load()
    cnt = lib.or_pair_set_rows(C.byref(osys.c), _ptr(x), box_inv, R, _ptr(rows), None, None, 0)
    pairs = np.zeros((max(cnt, 1), 2), np.int32)
    kind = np.zeros(max(cnt, 1), np.uint8)
    lib.or_pair_set_rows(C.byref(osys.c), _ptr(x), box_inv, R, _ptr(rows), _ptr(pairs), _ptr(kind), cnt)
    return pairs[:cnt], kind[:cnt]


def energy_forces(osys: OracleSystem, x: np.ndarray, lam: float) -> dict:
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    n = osys.spec.n
    terms = np.zeros(N_TERMS)
    F = np.zeros((n, 3))
    dl = np.zeros(3)
    dUdl = np.zeros(1)
    P = osys.n_theta
    dth = np.zeros(P)
    d2th = np.zeros(P)
    _load().or_energy_forces(C.byref(osys.c), _ptr(x), float(lam), _ptr(terms), _ptr(F), _ptr(dl),
                             _ptr(dUdl), _ptr(dth), _ptr(d2th))
    return dict(terms=terms, U=float(terms.sum()), F=F, dl=dl, dUdl=float(dUdl[0]), dth=dth,
                d2th=d2th)


def energy_forces_masked(osys: OracleSystem, x: np.ndarray, lam: float, atoms) -> dict:
    """Forces on `atoms` and dU/dlambda (complete); other forces and the
    energy terms are partial.  Visits only pairs touching a selected or an
    alchemical atom."""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    n = osys.spec.n
    mask = np.zeros(n, np.uint8)
    mask[np.asarray(atoms)] = 1
    terms = np.zeros(N_TERMS)
    F = np.zeros((n, 3))
    dl = np.zeros(3)
    dUdl = np.zeros(1)
    P = osys.n_theta
    dth, d2th = np.zeros(P), np.zeros(P)
    _load().or_energy_forces_masked(C.byref(osys.c), _ptr(x), float(lam), _ptr(mask), _ptr(terms), _ptr(F),
                                    _ptr(dl), _ptr(dUdl), _ptr(dth), _ptr(d2th))
    return dict(F=F, dl=dl, dUdl=float(dUdl[0]), dth=dth, d2th=d2th)


def set_threads(n: int) -> None:
    _load().or_set_threads(int(n))


def max_threads() -> int:
    return int(_load().or_get_max_threads())


def ti(sum_, count, lo, hi):
    nb = len(sum_)
    grad = np.zeros(nb)
    A = np.zeros(nb + 1)
    dA = np.zeros(1)
    s = np.ascontiguousarray(sum_, np.float64)
    c = np.ascontiguousarray(count, np.int64)
    _load().or_ti(_ptr(s), _ptr(c), nb, float(lo), float(hi), _ptr(grad), _ptr(A), _ptr(dA))
    return grad, A, float(dA[0])


class Simulation:
    """Multiple-walker lambda-ABF run of one system on the oracle."""

    def __init__(self, spec, run, state=None):
        from paper_2307_08006_gb300 import synth  # seeded inputs only

        self.spec, self.runspec = spec, run
        self.osys = OracleSystem(spec)
        st0 = state if state is not None else synth.initial_state(spec, run)
        W, n = run.n_walkers, spec.n
        P = self.osys.n_theta
        self.P = P
        nbins = [s.n_bins for s in run.stages]
        tot, mb = sum(nbins), max(nbins)
        self.stage_off = np.concatenate([[0], np.cumsum(nbins)]).astype(int)
        a = dict(
            walker_stage=run.walker_stage().astype(np.int32),
            x=np.ascontiguousarray(st0.x, np.float64).copy(),
            v=np.ascontiguousarray(st0.v, np.float64).copy(),
            lam=np.asarray(st0.lam, np.float64).copy(),
            plam=np.asarray(st0.plam, np.float64).copy(),
            step=np.zeros(W, np.uint64), F=np.zeros((W, n, 3)), G=np.zeros(W), s=np.zeros(W),
            dth=np.zeros((W, P)), d2th=np.zeros((W, P)),
            abf_sum=np.zeros(tot), abf_sumsq=np.zeros(tot), abf_count=np.zeros(tot, np.int64),
            dl_sum=np.zeros((W, mb)), dl_sumsq=np.zeros((W, mb)),
            dl_count=np.zeros((W, mb), np.int64),
            th_d2=np.zeros((tot, P)), th_d=np.zeros((tot, P)), th_sd=np.zeros((tot, P)))
        self.a = a
        st = _State()
        st.n_walkers = W
        for k, v in a.items():
            setattr(st, k, _ptr(v))
        self.st = st
        r = _Run()
        r.kT, r.dt, r.gamma = run.kT, run.dt, run.gamma
        r.m_lambda, r.gamma_lambda = run.m_lambda, run.gamma_lambda
        r.lambda_dynamics = int(run.lambda_dynamics)
        r.abf_on = int(run.abf_on)
        r.n_full = float(run.n_full)
        r.shared_freq = int(run.shared_freq)
        r.seed = int(run.seed) & 0xFFFFFFFF
        r.n_stages = len(run.stages)
        self._lo = np.asarray([s.lo for s in run.stages], np.float64)
        self._hi = np.asarray([s.hi for s in run.stages], np.float64)
        self._nb = np.asarray(nbins, np.int32)
        r.stage_lo, r.stage_hi, r.stage_bins = _ptr(self._lo), _ptr(self._hi), _ptr(self._nb)
        r.theta_stats = int(run.theta_stats)
        self.r = r
        self.lib = _load()
        self.lib.or_prime(C.byref(self.osys.c), C.byref(r), C.byref(st))

    def run(self, n_steps: int) -> None:
        self.lib.or_run(C.byref(self.osys.c), C.byref(self.r), C.byref(self.st), int(n_steps))

    def stage_bins(self, stage: int):
        o0, o1 = self.stage_off[stage], self.stage_off[stage + 1]
        return (self.a["abf_sum"][o0:o1].copy(), self.a["abf_sumsq"][o0:o1].copy(),
                self.a["abf_count"][o0:o1].copy())

    def delta_a(self, stage: int = 0):
        s, _, c = self.stage_bins(stage)
        st = self.runspec.stages[stage]
        return ti(s, c, st.lo, st.hi)

    def theta_gradient(self, stage: int = 0) -> np.ndarray:
        o0, o1 = self.stage_off[stage], self.stage_off[stage + 1]
        st = self.runspec.stages[stage]
        s, _, c = self.stage_bins(stage)
        out = np.zeros(self.P)
        arrs = [np.ascontiguousarray(self.a[k][o0:o1]) for k in ("th_d2", "th_d", "th_sd")]
        self.lib.or_theta_gradient(_ptr(s), _ptr(c), _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]),
                                   int(st.n_bins), float(st.lo), float(st.hi), int(self.P),
                                   float(self.runspec.kT), _ptr(out))
        return out
