"""The range-checked debug build (liblabf_checks.so, nvcc -DLA_CHECKS=1).

Every list, cell, slot and atom index that a kernel reads from device memory
is range-checked there before use; a failed check sets LA_STATUS_BAD_INDEX
(reported as LA_ERR_BAD_INDEX) and skips the access.  On valid systems no
check may fire and the results must be those of the release library: the
same pair sets (integer work, bit for bit) and the same forces, dU/dlambda
and trajectory.  The checked library runs in a child process (LABF_CHECKS=1
selects it there), so that each process loads one engine library.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT
from paper_2307_08006_gb300 import build as engine_build
from paper_2307_08006_gb300 import labf, synth

pytestmark = pytest.mark.gpu

# the same systems and steps in both processes
RUNNER = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2307_08006_gb300 import labf, synth
out = {}
sp = synth.water_box(137, 5, seed=5, box=1.7, r_cut=0.6)
rng = np.random.default_rng(5)
sp.x = ((sp.x + rng.normal(0, 0.03, sp.x.shape)) % sp.box).astype(np.float32)
run = synth.water_run(walkers_per_stage=2, n_bins=20)
st = synth.initial_state(sp, run, lam0=[0.1, 0.3, 0.6, 0.8])
inputs = [labf.SystemInput(sp, run, st)]
for k, s2 in enumerate(synth.uneven_batch(8008)[:3]):
    r2 = synth.uneven_run(seed=8008 + k, walkers_per_system=2)
    inputs.append(labf.SystemInput(s2, r2, synth.initial_state(s2, r2)))
eng = labf.Engine(inputs, options=dict(graph_steps=10, prune_margin=0.05))
w0 = 0
for i, si in enumerate(inputs):
    p, kind = eng.get_pairs(w0)
    out[f"pairs{i}"] = p
    out[f"kind{i}"] = kind
    ef = eng.energy_forces(w0)
    out[f"F{i}"] = ef["F"].cpu().numpy()
    out[f"dUdl{i}"] = np.array([ef["dUdl"]])
    w0 += si.run.n_walkers
eng.step(30)
out["x"] = np.concatenate([eng.get_state(w)["x"] for w in range(eng.n_walkers)])
out["lam"] = np.array([eng.get_state(w)["lam"] for w in range(eng.n_walkers)])
out["status"] = np.array([eng.sync()])
eng.close()
np.savez(sys.argv[2], **out)
"""


def _run(tmp_path, checks):
    script = tmp_path / "runner.py"
    script.write_text(RUNNER)
    out = tmp_path / ("checks.npz" if checks else "release.npz")
    env = dict(os.environ, LABF_CHECKS="1" if checks else "0")
    r = subprocess.run([sys.executable, str(script), ROOT, str(out)], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return dict(np.load(out))


def test_range_checked_build_reports_nothing_and_matches_release(tmp_path):
    assert os.path.exists(engine_build.build(checks=True))
    chk = _run(tmp_path, True)
    rel = _run(tmp_path, False)
    assert int(chk["status"][0]) == labf.LA_OK and int(rel["status"][0]) == labf.LA_OK
    for i in range(4):
        assert np.array_equal(chk[f"pairs{i}"], rel[f"pairs{i}"]), i
        assert np.array_equal(chk[f"kind{i}"], rel[f"kind{i}"]), i
        f, g = chk[f"F{i}"].astype(np.float64), rel[f"F{i}"].astype(np.float64)
        assert np.sqrt(((f - g) ** 2).sum() / (g ** 2).sum()) < 1e-6, i
        assert abs(chk[f"dUdl{i}"][0] - rel[f"dUdl{i}"][0]) <= 1e-6 * max(1.0, abs(rel[f"dUdl{i}"][0])), i
    # 30 steps: the trajectories agree to within FP32 rounding growth
    np.testing.assert_allclose(chk["x"], rel["x"], rtol=0, atol=1e-4)
    np.testing.assert_allclose(chk["lam"], rel["lam"], rtol=0, atol=1e-6)

