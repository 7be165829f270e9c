"""Python binding of liblabf (include/labf.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts
numpy/torch objects into the C ABI's pointers and back.  PyTorch provides
the device arena (one uint8 tensor) and the stream.  If the compiled
library is missing the import of :func:`load` raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

LA_OK = 0
LA_WARN_EMPTY_BIN = 1
LA_N_TERMS = 7
LA_PAIR_VARIANTS = 3
LA_MAX_WALKERS = 256
LA_N_STATS = 8
LA_N_KERNELS = 6
LA_EF_REBUILD = 0x1
LA_EF_COUNT_PAIRS = 0x2
TERM_NAMES = ("lj", "rf", "sc_lj", "sc_rf", "bond", "angle", "restraint")
KERNEL_NAMES = ("integrate", "rebuild", "pairs", "bonded", "walker", "lambda")
ERRORS = {-1: "INVALID_ARG", -2: "BOX_TOO_SMALL", -3: "CUDA", -4: "UNSUPPORTED", -5: "ARENA_TOO_SMALL",
          -6: "LIST_OVERFLOW", -7: "NONFINITE", -8: "FIXED_OVERFLOW", -9: "STATE", -10: "BAD_INDEX"}

EXPORTED = ("la_query_sizes", "la_create_system", "la_step_walkers", "la_step_walkers_plain",
            "la_read_abf", "la_abf_export", "la_abf_import", "la_energy_forces", "la_get_state", "la_set_state", "la_get_states", "la_set_states",
            "la_checkpoint_save", "la_checkpoint_load", "la_fp_peak", "la_energy_forces_device",
            "la_set_alch_params",
            "la_read_theta", "la_get_pairs", "la_lambda_path", "la_sync", "la_stats",
            "la_time_kernels", "la_autotune", "la_autotune_report", "la_last_error", "la_destroy",
            "la_alch_pairs_static", "la_static_last_error")


class LabfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"labf error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class la_system_desc(C.Structure):
    _fields_ = [
        ("n_atoms", C.c_int32), ("box", C.c_double),
        ("mass", C.c_void_p), ("charge", C.c_void_p), ("sigma", C.c_void_p), ("epsilon", C.c_void_p),
        ("alch", C.c_void_p), ("excl_group", C.c_void_p), ("excl_extra", C.c_void_p),
        ("n_bonds", C.c_int32), ("bond_ij", C.c_void_p), ("bond_r0", C.c_void_p), ("bond_k", C.c_void_p),
        ("n_angles", C.c_int32), ("angle_ijk", C.c_void_p), ("angle_t0", C.c_void_p),
        ("angle_k", C.c_void_p),
        ("n_posres", C.c_int32), ("posres_idx", C.c_void_p), ("posres_x0", C.c_void_p),
        ("posres_k", C.c_double),
        ("n_fb_a", C.c_int32), ("fb_a", C.c_void_p), ("n_fb_b", C.c_int32), ("fb_b", C.c_void_p),
        ("fb_d0", C.c_double), ("fb_k", C.c_double),
        ("n_lh", C.c_int32), ("lh_idx", C.c_void_p), ("lh_x0", C.c_void_p),
        ("lh_k0", C.c_double), ("lh_k1", C.c_double), ("lh_dims", C.c_int32),
        ("r_cut", C.c_double), ("eps_rf", C.c_double), ("coul", C.c_double),
        ("b_v", C.c_double), ("b_e", C.c_double), ("sc_alpha", C.c_double),
        ("sc_n", C.c_int32), ("sc_m", C.c_int32),
        ("kT", C.c_double), ("dt", C.c_double), ("gamma", C.c_double), ("m_lambda", C.c_double),
        ("gamma_lambda", C.c_double), ("skin", C.c_double), ("n_full", C.c_double),
        ("shared_freq", C.c_int32), ("seed", C.c_uint32),
        ("lambda_dynamics", C.c_int32), ("abf_on", C.c_int32), ("theta_stats", C.c_int32),
        ("n_stages", C.c_int32),
        ("stage_lo", C.c_void_p), ("stage_hi", C.c_void_p), ("stage_bins", C.c_void_p),
        ("stage_walkers", C.c_void_p),
        ("x0", C.c_void_p), ("v0", C.c_void_p), ("lam0", C.c_void_p), ("plam0", C.c_void_p),
        ("n_lr", C.c_int32), ("lr_ij", C.c_void_p), ("lr_delta", C.c_double), ("lr_k", C.c_double),
    ]


class la_options(C.Structure):
    _fields_ = [("graph_steps", C.c_int32), ("autotune", C.c_int32),
                ("list_capacity_factor", C.c_double), ("pair_variant", C.c_int32),
                ("pair_ctas_per_sm", C.c_int32), ("chunk_entries", C.c_int32),
                ("prune_margin", C.c_double)]


_lib = None


def lib_path() -> str:
    """The engine library; with LABF_CHECKS=1 in the environment, the
    range-checked debug build (every index read from a device list is
    checked; a bad one is reported as LA_ERR_BAD_INDEX)."""
    return _build.LIB_CHECKS if os.environ.get("LABF_CHECKS") == "1" else _build.LIB


def load(build_if_missing: bool = False):
    """Load liblabf.so.  Raises if it is missing (no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"liblabf.so not built at {path}: run __graft_entry__.build()")
        _build.build(checks=path == _build.LIB_CHECKS)
    lib = C.CDLL(path)
    P, I, D, S = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    H = C.c_void_p
    lib.la_query_sizes.argtypes = [P, I, P, C.POINTER(S)]
    lib.la_create_system.argtypes = [P, I, P, P, S, P, C.POINTER(H)]
    lib.la_step_walkers.argtypes = [H, C.c_int64, P]
    lib.la_step_walkers_plain.argtypes = [H, C.c_int64, P]
    lib.la_read_abf.argtypes = [H, I, I, P, P, P, P, P, P, P, P]
    lib.la_abf_export.argtypes = [H, I, I, P, P, P, P]
    lib.la_abf_import.argtypes = [H, I, I, P, P, P, P]
    lib.la_energy_forces.argtypes = [H, I, C.c_uint32, P, P, P, P, P, P]
    lib.la_get_state.argtypes = [H, I, P, P, P, P, P, P]
    lib.la_set_state.argtypes = [H, I, P, P, P, P, P, P]
    lib.la_get_states.argtypes = [H, P, P, P, P, P, P]
    lib.la_set_states.argtypes = [H, P, P, P, P, P, P]
    lib.la_checkpoint_save.argtypes = [H, P, S, C.POINTER(S), P]
    lib.la_checkpoint_load.argtypes = [H, P, S, P]
    lib.la_fp_peak.argtypes = [I, D, C.POINTER(D), P]
    lib.la_energy_forces_device.argtypes = [H, I, P, P, P, P, P, P]
    lib.la_set_alch_params.argtypes = [H, I, P, P]
    lib.la_read_theta.argtypes = [H, I, I, P, P, P, P, P]
    lib.la_get_pairs.argtypes = [H, I, P, P, C.c_int64, P, P]
    lib.la_lambda_path.argtypes = [H, P, I, D, D, P, P]
    lib.la_sync.argtypes = [H, P, P]
    lib.la_stats.argtypes = [H, P, P]
    lib.la_time_kernels.argtypes = [H, I, P, P, P]
    lib.la_autotune.argtypes = [H, P]
    lib.la_autotune_report.argtypes = [H]
    lib.la_autotune_report.restype = C.c_char_p
    lib.la_last_error.argtypes = [H]
    lib.la_last_error.restype = C.c_char_p
    lib.la_destroy.argtypes = [H]
    lib.la_alch_pairs_static.argtypes = [I, P, P, P, P, P, P, I, P, D, D, D, D, D, D, D, D, I, I, P, P, P]
    lib.la_static_last_error.argtypes = []
    lib.la_static_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("la_autotune_report", "la_last_error", "la_static_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _Keep:
    """Holds numpy arrays referenced by a descriptor until create returns."""

    def __init__(self):
        self.items = []

    def arr(self, a, dt, shape=None):
        a = np.ascontiguousarray(a, dtype=dt)
        if shape is not None:
            a = a.reshape(shape)
        self.items.append(a)
        return _p(a) if a.size else None


def make_desc(spec, run, state, keep: _Keep) -> la_system_desc:
    """Marshal a SystemSpec / RunSpec / WalkerState into la_system_desc."""
    d = la_system_desc()
    k = keep
    d.n_atoms = spec.n
    d.box = float(spec.box)
    d.mass = k.arr(spec.mass, np.float64)
    d.charge = k.arr(spec.charge, np.float64)
    d.sigma = k.arr(spec.sigma, np.float64)
    d.epsilon = k.arr(spec.epsilon, np.float64)
    d.alch = k.arr(spec.alch, np.uint8)
    d.excl_group = k.arr(spec.excl_group, np.int32)
    d.excl_extra = k.arr(spec.excl_extra, np.int32)
    d.n_bonds = len(spec.bond_r0)
    d.bond_ij = k.arr(spec.bond_ij, np.int32)
    d.bond_r0 = k.arr(spec.bond_r0, np.float64)
    d.bond_k = k.arr(spec.bond_k, np.float64)
    d.n_angles = len(spec.angle_t0)
    d.angle_ijk = k.arr(spec.angle_ijk, np.int32)
    d.angle_t0 = k.arr(spec.angle_t0, np.float64)
    d.angle_k = k.arr(spec.angle_k, np.float64)
    d.n_posres = len(spec.posres_idx)
    d.posres_idx = k.arr(spec.posres_idx, np.int32)
    d.posres_x0 = k.arr(spec.posres_x0, np.float64)
    d.posres_k = float(spec.posres_k)
    d.n_fb_a, d.fb_a = len(spec.fb_a), k.arr(spec.fb_a, np.int32)
    d.n_fb_b, d.fb_b = len(spec.fb_b), k.arr(spec.fb_b, np.int32)
    d.fb_d0, d.fb_k = float(spec.fb_d0), float(spec.fb_k)
    d.n_lh, d.lh_idx = len(spec.lh_idx), k.arr(spec.lh_idx, np.int32)
    d.lh_x0 = k.arr(spec.lh_x0, np.float64)
    d.lh_k0, d.lh_k1, d.lh_dims = float(spec.lh_k0), float(spec.lh_k1), int(spec.lh_dims)
    d.r_cut, d.eps_rf, d.coul = float(spec.r_cut), float(spec.eps_rf), float(spec.coul)
    d.b_v, d.b_e, d.sc_alpha = float(spec.b_v), float(spec.b_e), float(spec.sc_alpha)
    d.sc_n, d.sc_m = int(spec.sc_n), int(spec.sc_m)
    d.kT, d.dt, d.gamma = float(run.kT), float(run.dt), float(run.gamma)
    d.m_lambda, d.gamma_lambda = float(run.m_lambda), float(run.gamma_lambda)
    d.skin, d.n_full = float(run.skin), float(run.n_full)
    d.shared_freq, d.seed = int(run.shared_freq), int(run.seed) & 0xFFFFFFFF
    d.lambda_dynamics, d.abf_on = int(run.lambda_dynamics), int(run.abf_on)
    d.theta_stats = int(run.theta_stats)
    d.n_stages = len(run.stages)
    d.stage_lo = k.arr([s.lo for s in run.stages], np.float64)
    d.stage_hi = k.arr([s.hi for s in run.stages], np.float64)
    d.stage_bins = k.arr([s.n_bins for s in run.stages], np.int32)
    d.stage_walkers = k.arr([s.n_walkers for s in run.stages], np.int32)
    d.x0 = k.arr(state.x, np.float32)
    d.v0 = k.arr(state.v, np.float32)
    d.lam0 = k.arr(state.lam, np.float64)
    d.plam0 = k.arr(state.plam, np.float64)
    d.n_lr = len(spec.lr_ij)
    d.lr_ij = k.arr(np.asarray(spec.lr_ij).reshape(-1, 2), np.int32)
    d.lr_delta, d.lr_k = float(spec.lr_delta), float(spec.lr_k)
    return d


@dataclass
class SystemInput:
    spec: object
    run: object
    state: object


class Engine:
    """An engine instance over one or more systems (their walkers batched).

    The device arena is one torch uint8 tensor; all device work goes on the
    current torch stream of the arena's device unless a stream is given.
    """

    def __init__(self, systems: Sequence[SystemInput], options: Optional[dict] = None,
                 device: int = 0):
        import torch

        self.torch = torch
        self.lib = load()
        self.systems = list(systems)
        keep = _Keep()
        descs = (la_system_desc * len(self.systems))()
        for i, s in enumerate(self.systems):
            descs[i] = make_desc(s.spec, s.run, s.state, keep)
        opt = la_options()
        for k, v in (options or {}).items():
            setattr(opt, k, v)
        self._opt = opt
        nbytes = C.c_size_t(0)
        self._check(self.lib.la_query_sizes(C.cast(descs, C.c_void_p), len(descs), C.byref(opt),
                                            C.byref(nbytes)), None)
        self.device = torch.device("cuda", device)
        self.arena = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        self.handle = C.c_void_p()
        rc = self.lib.la_create_system(C.cast(descs, C.c_void_p), len(descs), C.byref(opt),
                                       C.c_void_p(self.arena.data_ptr()), nbytes, self._stream(),
                                       C.byref(self.handle))
        self._check(rc)
        del keep
        self.walker_sys, self.walker_local = [], []
        for si, s in enumerate(self.systems):
            for wl in range(s.run.n_walkers):
                self.walker_sys.append(si)
                self.walker_local.append(wl)
        self.n_walkers = len(self.walker_sys)
        # first row of each walker in the all-walker state arrays
        sizes = [self.systems[si].spec.n for si in self.walker_sys]
        self.walker_rows = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)

    # -- plumbing -------------------------------------------------------
    def _stream(self, stream=None):
        if stream is None:
            stream = self.torch.cuda.current_stream(self.device)
        return C.c_void_p(stream.cuda_stream)

    def _check(self, rc, handle="self"):
        if rc < 0:
            h = self.handle if handle == "self" else None
            msg = self.lib.la_last_error(h).decode() if h else ""
            raise LabfError(rc, msg)
        return rc

    def close(self):
        if getattr(self, "handle", None):
            self.lib.la_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- stepping ---------------------------------------------------------
    def step(self, n_steps: int, stream=None):
        self._check(self.lib.la_step_walkers(self.handle, int(n_steps), self._stream(stream)))

    def step_plain(self, n_steps: int, stream=None):
        self._check(self.lib.la_step_walkers_plain(self.handle, int(n_steps), self._stream(stream)))

    def sync(self, stream=None) -> int:
        bits = C.c_uint32(0)
        self._check(self.lib.la_sync(self.handle, self._stream(stream), C.byref(bits)))
        return int(bits.value)

    # -- read-outs --------------------------------------------------------
    def read_abf(self, sys: int = 0, stage: int = 0, stream=None) -> dict:
        nb = self.systems[sys].run.stages[stage].n_bins
        s1, s2, A = np.zeros(nb), np.zeros(nb), np.zeros(nb + 1)
        cnt = np.zeros(nb, np.int64)
        grad = np.zeros(nb)
        dA, se = C.c_double(0), C.c_double(0)
        rc = self.lib.la_read_abf(self.handle, sys, stage, _p(s1), _p(s2), _p(cnt), _p(grad), _p(A),
                                  C.byref(dA), C.byref(se), self._stream(stream))
        self._check(rc)
        return dict(sum=s1, sumsq=s2, count=cnt, grad=grad, A=A, dA=dA.value, dA_se=se.value,
                    empty_bin=rc == LA_WARN_EMPTY_BIN)

    def abf_export(self, sys: int = 0, stage: int = 0, stream=None):
        """Unmerged bin statistics of the stage's walkers, summed in walker order."""
        nb = self.systems[sys].run.stages[stage].n_bins
        s1, s2, cnt = np.zeros(nb), np.zeros(nb), np.zeros(nb, np.int64)
        self._check(self.lib.la_abf_export(self.handle, sys, stage, _p(s1), _p(s2), _p(cnt),
                                           self._stream(stream)))
        return s1, s2, cnt

    def abf_import(self, sum, sumsq, count, sys: int = 0, stage: int = 0, stream=None) -> None:
        """Add host totals to the shared statistics; clears the unmerged ones."""
        nb = self.systems[sys].run.stages[stage].n_bins
        s1 = np.ascontiguousarray(sum, np.float64)
        s2 = np.ascontiguousarray(sumsq, np.float64)
        cnt = np.ascontiguousarray(count, np.int64)
        if s1.shape != (nb,) or s2.shape != (nb,) or cnt.shape != (nb,):
            raise ValueError(f"abf_import wants [{nb}] arrays")
        self._check(self.lib.la_abf_import(self.handle, sys, stage, _p(s1), _p(s2), _p(cnt),
                                           self._stream(stream)))

    def energy_forces(self, walker: int, rebuild: bool = False, count_pairs: bool = False,
                      forces: bool = True, stream=None) -> dict:
        si = self.walker_sys[walker]
        spec = self.systems[si].spec
        P = 3 * spec.n_alch + 1
        terms = np.zeros(LA_N_TERMS)
        dudl = C.c_double(0)
        dth, d2 = np.zeros(P), np.zeros(P)
        f = self.torch.zeros((spec.n, 3), dtype=self.torch.float32, device=self.device) if forces else None
        flags = (LA_EF_REBUILD if rebuild else 0) | (LA_EF_COUNT_PAIRS if count_pairs else 0)
        self._check(self.lib.la_energy_forces(self.handle, walker, flags, _p(terms),
                                              C.c_void_p(f.data_ptr()) if f is not None else None,
                                              C.byref(dudl), _p(dth), _p(d2), self._stream(stream)))
        out = dict(terms=terms, U=float(terms.sum()), dUdl=dudl.value, dth=dth, d2th=d2, F=f)
        if count_pairs:
            st = self.stats(stream)
            out["pairs_normal"], out["pairs_alch"] = int(st[3]), int(st[4])
        return out

    def energy_forces_device(self, walker: int, x=None, theta=None, lam=None, out=None, forces=None,
                             stream=None) -> None:
        """la_energy_forces_device: every argument a CUDA tensor (or None) on
        the engine's device; x float32 [n, 3], theta float64 [n_alch, 3],
        lam float64 [1], out float64 [LA_N_TERMS + 2 + 2 P], forces float32
        [n, 3].  Asynchronous (no host synchronisation)."""
        def ptr(t, dtype, numel=None):
            if t is None:
                return None
            if t.device != self.device or t.dtype != dtype or not t.is_contiguous():
                raise ValueError(f"expected a contiguous {dtype} tensor on {self.device}")
            if numel is not None and t.numel() != numel:
                raise ValueError(f"expected {numel} elements, got {t.numel()}")
            return C.c_void_p(t.data_ptr())

        spec = self.systems[self.walker_sys[walker]].spec
        P = 3 * spec.n_alch + 1
        self._check(self.lib.la_energy_forces_device(
            self.handle, walker, ptr(x, self.torch.float32, 3 * spec.n), ptr(theta, self.torch.float64, 3 * spec.n_alch),
            ptr(lam, self.torch.float64, 1), ptr(out, self.torch.float64, LA_N_TERMS + 2 + 2 * P),
            ptr(forces, self.torch.float32, 3 * spec.n), self._stream(stream)))

    def get_state(self, walker: int, stream=None) -> dict:
        n = self.systems[self.walker_sys[walker]].spec.n
        x, v = np.zeros((n, 3), np.float32), np.zeros((n, 3), np.float32)
        lam, plam, step = C.c_double(0), C.c_double(0), C.c_uint64(0)
        self._check(self.lib.la_get_state(self.handle, walker, _p(x), _p(v), C.byref(lam), C.byref(plam),
                                          C.byref(step), self._stream(stream)))
        return dict(x=x, v=v, lam=lam.value, plam=plam.value, step=step.value)

    def set_state(self, walker: int, x=None, v=None, lam=None, plam=None, step=None, stream=None):
        xa = None if x is None else np.ascontiguousarray(x, np.float32)
        va = None if v is None else np.ascontiguousarray(v, np.float32)
        la = None if lam is None else C.byref(C.c_double(float(lam)))
        pa = None if plam is None else C.byref(C.c_double(float(plam)))
        sa = None if step is None else C.byref(C.c_uint64(int(step)))
        self._check(self.lib.la_set_state(self.handle, walker, _p(xa), _p(va), la, pa, sa, self._stream(stream)))

    def _rows_array(self, a, name):
        n = int(self.walker_rows[-1])
        if a.dtype != np.float32 or a.shape != (n, 3) or not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name}: expected a C-contiguous float32 array of shape ({n}, 3)")
        return a

    def _pinned(self, shape, dtype):
        """A numpy view of a page-locked host tensor (copied by DMA)."""
        t = self.torch.empty(shape, dtype=dtype, pin_memory=True)
        self._pin_keep = getattr(self, "_pin_keep", [])[-8:] + [t]
        return t.numpy()

    def get_states(self, x=None, v=None, stream=None) -> dict:
        """Every walker's state in one call.  x, v: float32 [rows, 3], walker w
        in rows walker_rows[w]:walker_rows[w + 1]; arrays passed in (e.g.
        views of page-locked tensors) are filled in place, otherwise
        page-locked arrays are allocated, so that the call synchronises
        once.  Also returns every walker's step counter."""
        n = int(self.walker_rows[-1])
        x = self._pinned((n, 3), self.torch.float32) if x is None else self._rows_array(x, "x")
        v = self._pinned((n, 3), self.torch.float32) if v is None else self._rows_array(v, "v")
        lam, plam = np.zeros(self.n_walkers), np.zeros(self.n_walkers)
        step = np.zeros(self.n_walkers, np.uint64)
        self._check(self.lib.la_get_states(self.handle, _p(x), _p(v), _p(lam), _p(plam), _p(step),
                                           self._stream(stream)))
        return dict(x=x, v=v, lam=lam, plam=plam, step=step)

    def set_states(self, x=None, v=None, lam=None, plam=None, step=None, stream=None):
        """Every walker's state in one call (layout as in get_states); step
        sets the walkers' step counters (the Philox counters)."""
        xa = None if x is None else self._rows_array(x, "x")
        va = None if v is None else self._rows_array(v, "v")
        la = None if lam is None else np.ascontiguousarray(lam, np.float64).reshape(self.n_walkers)
        pa = None if plam is None else np.ascontiguousarray(plam, np.float64).reshape(self.n_walkers)
        sa = None if step is None else np.ascontiguousarray(step, np.uint64).reshape(self.n_walkers)
        self._check(self.lib.la_set_states(self.handle, _p(xa), _p(va), _p(la), _p(pa), _p(sa),
                                           self._stream(stream)))

    def checkpoint(self, stream=None) -> np.ndarray:
        """The engine's complete state as a byte image (page-locked uint8
        array): la_checkpoint_save.  Restore with load_checkpoint into an
        engine created from the same inputs and options."""
        n = C.c_size_t(0)
        self._check(self.lib.la_checkpoint_save(self.handle, None, 0, C.byref(n), self._stream(stream)))
        buf = self.torch.empty(int(n.value), dtype=self.torch.uint8, pin_memory=True).numpy()
        self._check(self.lib.la_checkpoint_save(self.handle, _p(buf), buf.size, C.byref(n), self._stream(stream)))
        return buf

    def load_checkpoint(self, image: np.ndarray, stream=None) -> None:
        img = np.ascontiguousarray(image, np.uint8)
        self._check(self.lib.la_checkpoint_load(self.handle, _p(img), img.size, self._stream(stream)))

    def set_alch_params(self, sys: int, theta: np.ndarray, stream=None):
        t = np.ascontiguousarray(theta, np.float64)
        self._check(self.lib.la_set_alch_params(self.handle, sys, _p(t), self._stream(stream)))

    def read_theta(self, sys: int = 0, stage: int = 0, stream=None) -> dict:
        spec = self.systems[sys].spec
        nb = self.systems[sys].run.stages[stage].n_bins
        P = 3 * spec.n_alch + 1
        a, b, c = np.zeros((nb, P)), np.zeros((nb, P)), np.zeros((nb, P))
        g = np.zeros(P)
        rc = self._check(self.lib.la_read_theta(self.handle, sys, stage, _p(a), _p(b), _p(c), _p(g),
                                                self._stream(stream)))
        return dict(sum_d2=a, sum_d=b, sum_sd=c, dA_dtheta=g, empty_bin=rc == LA_WARN_EMPTY_BIN)

    def get_pairs(self, walker: int, stream=None) -> Tuple[np.ndarray, np.ndarray]:
        cnt = C.c_int64(0)
        self._check(self.lib.la_get_pairs(self.handle, walker, None, None, 0, C.byref(cnt), self._stream(stream)))
        n = int(cnt.value)
        pairs = np.zeros((max(n, 1), 2), np.int32)
        kind = np.zeros(max(n, 1), np.uint8)
        self._check(self.lib.la_get_pairs(self.handle, walker, _p(pairs), _p(kind), n, C.byref(cnt),
                                          self._stream(stream)))
        return pairs[:n], kind[:n]

    def lambda_path(self, lam: np.ndarray, b_v: float, b_e: float, stream=None) -> np.ndarray:
        lam = np.ascontiguousarray(lam, np.float64)
        out = np.zeros((lam.size, 4))
        self._check(self.lib.la_lambda_path(self.handle, _p(lam), lam.size, float(b_v), float(b_e), _p(out),
                                            self._stream(stream)))
        return out

    def stats(self, stream=None) -> np.ndarray:
        out = np.zeros(LA_N_STATS, np.int64)
        self._check(self.lib.la_stats(self.handle, _p(out), self._stream(stream)))
        return out

    def time_kernels(self, n_steps: int, stream=None) -> dict:
        ms = np.zeros(LA_N_KERNELS, np.float32)
        cnt = np.zeros(LA_N_KERNELS, np.int64)
        self._check(self.lib.la_time_kernels(self.handle, int(n_steps), _p(ms), _p(cnt), self._stream(stream)))
        return {k: (float(m), int(c)) for k, m, c in zip(KERNEL_NAMES, ms, cnt)}

    def autotune(self, stream=None) -> str:
        """Re-tune the pair kernel's launch shape on the current lists."""
        self._check(self.lib.la_autotune(self.handle, self._stream(stream)))
        return self.autotune_report()

    def autotune_report(self) -> str:
        return self.lib.la_autotune_report(self.handle).decode()


def fp_peak(fp64: bool = False, seconds: float = 0.5, stream=None) -> float:
    """Measured FMA rate of the current GPU in TFLOP/s (la_fp_peak)."""
    import torch

    lib = load()
    out = C.c_double(0.0)
    st = torch.cuda.current_stream() if stream is None else stream
    rc = lib.la_fp_peak(1 if fp64 else 0, float(seconds), C.byref(out), C.c_void_p(st.cuda_stream))
    if rc < 0:
        raise LabfError(rc, "la_fp_peak failed")
    return out.value


def engine_for(spec, run, state=None, options=None) -> Engine:
    """One-system convenience constructor."""
    from . import synth

    st = state if state is not None else synth.initial_state(spec, run)
    return Engine([SystemInput(spec, run, st)], options)


def alch_pairs_static(x, q, sigma, epsilon, alch, excl_group, alch_idx, box, r_cut, eps_rf, coul, lam,
                      b_v, b_e, sc_alpha=0.5, sc_n=1, sc_m=1, forces=None, out=None, stream=None):
    """Marshal torch CUDA tensors into la_alch_pairs_static (no allocation
    in the library; `forces` [n, 3] float32 and `out` [6] float64 may be
    passed pre-allocated).  out = (dU/dlambda, dU/dlambda_v, dU/dlambda_e,
    soft-core LJ energy, lambda_e RF energy, device status bits)."""
    import torch

    lib = load()
    n = int(x.shape[0])
    if forces is None:
        forces = torch.empty((n, 3), dtype=torch.float32, device=x.device)
    if out is None:
        out = torch.empty(6, dtype=torch.float64, device=x.device)
    if tuple(forces.shape) != (n, 3) or out.numel() < 6:
        raise ValueError("alch_pairs_static wants forces [n, 3] and out [6]")
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    ptr = lambda t: C.c_void_p(t.data_ptr())
    rc = lib.la_alch_pairs_static(n, ptr(x), ptr(q), ptr(sigma), ptr(epsilon), ptr(alch), ptr(excl_group),
                                  int(alch_idx.numel()), ptr(alch_idx), float(box), float(r_cut), float(eps_rf),
                                  float(coul), float(lam), float(b_v), float(b_e), float(sc_alpha), int(sc_n),
                                  int(sc_m), ptr(forces), ptr(out), C.c_void_p(stream.cuda_stream))
    if rc < 0:
        raise LabfError(rc, lib.la_static_last_error().decode())
    return forces, out
