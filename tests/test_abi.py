"""The C-ABI library builds, loads without a GPU and exports every symbol
that include/labf.h declares; descriptor layouts agree with the header."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT
from paper_2307_08006_gb300 import build as engine_build
from paper_2307_08006_gb300 import labf, synth


def _declared():
    src = open(os.path.join(ROOT, "include", "labf.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(la_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol():
    lib = engine_build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (la_\w+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    assert set(declared) == set(labf.EXPORTED)


def test_library_loads_without_gpu():
    lib = labf.load(build_if_missing=True)
    for name in labf.EXPORTED:
        assert hasattr(lib, name)


def test_binding_constants_match_header():
    src = open(os.path.join(ROOT, "include", "labf.h")).read()
    defs = {m.group(1): m.group(2) for m in re.finditer(r"^#define (LA_\w+) (\S+)", src, re.M)}
    for name in ("LA_OK", "LA_WARN_EMPTY_BIN", "LA_N_TERMS", "LA_PAIR_VARIANTS", "LA_MAX_WALKERS", "LA_N_STATS",
                 "LA_N_KERNELS", "LA_EF_REBUILD", "LA_EF_COUNT_PAIRS"):
        assert int(defs[name].rstrip("u"), 0) == getattr(labf, name), name
    for name, v in defs.items():
        if name.startswith("LA_ERR_"):
            code = int(v.strip("()"))
            assert labf.ERRORS[code] == name[len("LA_ERR_"):], name


def test_descriptor_layout_matches_header(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "labf.h"\n'
                    'int main(){printf("%zu %zu %zu %zu %zu\\n", sizeof(la_system_desc),'
                    ' offsetof(la_system_desc, kT), offsetof(la_system_desc, plam0),'
                    ' offsetof(la_system_desc, seed), sizeof(la_options));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    D = labf.la_system_desc
    assert got == [C.sizeof(D), D.kT.offset, D.plam0.offset, D.seed.offset, C.sizeof(labf.la_options)]


def _query(spec, run, state=None, opt=None):
    lib = labf.load(build_if_missing=True)
    keep = labf._Keep()
    st = state if state is not None else synth.initial_state(spec, run)
    d = labf.make_desc(spec, run, st, keep)
    n = C.c_size_t(0)
    rc = lib.la_query_sizes(C.byref(d), 1, opt, C.byref(n))
    return rc, n.value


def test_query_sizes_host_only():
    rc, n = _query(synth.lj_fluid(), synth.lj_fluid_run())
    assert rc == 0 and n > 0 and n % 256 == 0
    rc2, n2 = _query(synth.water_box(), synth.water_run())
    assert rc2 == 0 and n2 > n


def test_query_rejects_bad_input():
    sp = synth.water_box(64, 4, box=1.25, r_cut=0.5)
    run = synth.water_run(walkers_per_stage=1)
    assert _query(sp, run)[0] == 0
    # box smaller than twice the list radius
    small = synth.with_changes(sp, r_cut=0.6)
    assert _query(small, run)[0] == -2
    # non-positive mass, out-of-range bond index, empty stage list
    bad = synth.with_changes(sp, mass=np.where(np.arange(sp.n) == 3, 0.0, sp.mass))
    assert _query(bad, run)[0] == -1
    bi = sp.bond_ij.copy()
    bi[0, 1] = sp.n
    assert _query(synth.with_changes(sp, bond_ij=bi), run)[0] == -1
    run0 = synth.water_run(walkers_per_stage=1)
    run0.stages = []
    assert _query(sp, run0)[0] == -1
    # a stage without walkers or bins, an empty lambda interval, a negative
    # shared_freq
    for field, value in (("n_walkers", 0), ("n_bins", 0), ("hi", 0.0)):
        r = synth.water_run(walkers_per_stage=1)
        setattr(r.stages[1], field, value)
        assert _query(sp, r)[0] == -1, field
    r = synth.water_run(walkers_per_stage=1)
    r.shared_freq = -1
    assert _query(sp, r)[0] == -1


def test_walker_limit():
    """At most 256 walkers per handle (the pair kernel's per-walker prefix
    sums live in shared memory)."""
    sp = synth.lj_fluid()
    assert _query(sp, synth.lj_fluid_run(n_walkers=256))[0] == 0
    assert _query(sp, synth.lj_fluid_run(n_walkers=257))[0] == -1


def test_calls_reject_a_null_handle():
    """Every handle call returns LA_ERR_INVALID_ARG for a NULL handle without
    touching the device (no GPU needed)."""
    lib = labf.load()
    x = np.zeros((4, 3), np.float32)
    lam = np.zeros(2)
    assert lib.la_get_states(None, labf._p(x), labf._p(x), labf._p(lam), labf._p(lam), None, None) == -1
    assert lib.la_set_states(None, labf._p(x), labf._p(x), labf._p(lam), labf._p(lam), None, None) == -1
    assert lib.la_get_state(None, 0, labf._p(x), labf._p(x), None, None, None, None) == -1
    assert lib.la_set_state(None, 0, labf._p(x), labf._p(x), None, None, None, None) == -1
    n = C.c_size_t(0)
    assert lib.la_checkpoint_save(None, None, 0, C.byref(n), None) == -1
    assert lib.la_checkpoint_load(None, labf._p(x), 16, None) == -1
    assert lib.la_step_walkers(None, 1, None) == -1


def test_soft_core_powers_below_one_are_rejected():
    """n lambda_v^(n-1) at lambda_v = 0 and m (1 - lambda_v)^(m-1) at
    lambda_v = 1 are 0 * inf for powers 0, so the soft-core family is
    n, m >= 1: la_query_sizes and la_alch_pairs_static both reject smaller
    powers on the host, before any device work."""
    sp = synth.water_box(64, 4, box=1.25, r_cut=0.5)
    run = synth.water_run(walkers_per_stage=1)
    assert _query(synth.with_changes(sp, sc_n=1, sc_m=1), run)[0] == 0
    assert _query(synth.with_changes(sp, sc_n=2, sc_m=2), run)[0] == 0
    assert _query(synth.with_changes(sp, sc_n=0), run)[0] == -1
    assert _query(synth.with_changes(sp, sc_m=0), run)[0] == -1
    lib = labf.load()
    buf = np.zeros(16, np.float64)  # never read: the call fails during validation
    p = labf._p(buf)
    for n_, m_ in ((0, 1), (1, 0), (-1, 1)):
        rc = lib.la_alch_pairs_static(4, p, p, p, p, p, p, 1, p, 10.0, 1.0, 78.0, 1.0, 0.5, 0.5, 0.5, 0.5,
                                      n_, m_, p, p, None)
        assert rc == -1
        assert b"soft-core powers" in lib.la_static_last_error()


def test_oracle_rejects_soft_core_powers_below_one():
    import oracle

    sp = synth.water_box(64, 4, box=1.25, r_cut=0.5)
    oracle.OracleSystem(synth.with_changes(sp, sc_n=2, sc_m=1))
    for kw in (dict(sc_n=0), dict(sc_m=0)):
        with pytest.raises(ValueError, match="soft-core powers"):
            oracle.OracleSystem(synth.with_changes(sp, **kw))
