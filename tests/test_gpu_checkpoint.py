"""Exact restarts: la_checkpoint_save / la_checkpoint_load and the step
counters of la_get_states / la_set_states, through the C ABI on the GPU.

A run continued from a checkpoint in a fresh engine (created from the same
inputs and options) must equal the uninterrupted run bit for bit: positions,
velocities, lambda, p_lambda, step counters (the Philox counters, SI S1 noise)
and the ABF accumulators of every stage (Sec. 2.3, 2.4).
"""
import numpy as np
import pytest

from paper_2307_08006_gb300 import labf, synth

pytestmark = pytest.mark.gpu


def _inputs(seed=501):
    sp = synth.water_box(256, 4, seed=seed, r_cut=0.85)
    rng = np.random.default_rng(seed)
    sp.x = ((sp.x + rng.normal(0.0, 0.01, sp.x.shape)) % sp.box).astype(np.float32)
    run = synth.water_run(seed=seed + 1, walkers_per_stage=2, n_bins=20)
    return sp, run, synth.initial_state(sp, run, lam0=[0.1, 0.3, 0.6, 0.9])


def _engine(sp, run, st, **opt):
    o = dict(graph_steps=10, prune_margin=0.05)
    o.update(opt)
    return labf.Engine([labf.SystemInput(sp, run, st)], options=o)


def _snapshot(eng, run):
    s = eng.get_states()
    abf = [eng.read_abf(0, k) for k in range(len(run.stages))]
    return s, abf


def _assert_same(a, b):
    (sa, aa), (sb, ab) = a, b
    for k in ("x", "v", "lam", "plam", "step"):
        assert np.array_equal(np.asarray(sa[k]), np.asarray(sb[k])), k
    for ra, rb in zip(aa, ab):
        assert np.array_equal(ra["count"], rb["count"])
        assert np.array_equal(ra["sum"], rb["sum"]) and np.array_equal(ra["sumsq"], rb["sumsq"])


def test_checkpoint_restart_is_bit_exact():
    sp, run, st = _inputs()
    full = _engine(sp, run, st)
    full.step(40)
    ref = _snapshot(full, run)
    full.close()

    first = _engine(sp, run, st)
    first.step(20)
    image = first.checkpoint()
    mid = _snapshot(first, run)
    first.close()
    assert int(np.asarray(mid[0]["step"]).min()) == 20

    resumed = _engine(sp, run, st)
    resumed.step(3)  # state that the load must overwrite entirely
    resumed.load_checkpoint(image)
    _assert_same(_snapshot(resumed, run), mid)
    resumed.step(20)
    _assert_same(_snapshot(resumed, run), ref)
    # the one-walker-per-launch form continues the same way from the image
    plain = _engine(sp, run, st)
    plain.load_checkpoint(image)
    plain.step_plain(20)
    _assert_same(_snapshot(plain, run), ref)
    resumed.close()
    plain.close()


def test_checkpoint_of_another_system_is_refused():
    sp, run, st = _inputs()
    a = _engine(sp, run, st)
    a.step(5)
    image = a.checkpoint()
    other = synth.water_run(seed=run.seed + 7, walkers_per_stage=2, n_bins=20)  # another seed
    b = _engine(sp, other, synth.initial_state(sp, other, lam0=[0.1, 0.3, 0.6, 0.9]))
    before = b.get_states()
    with pytest.raises(labf.LabfError, match="different"):
        b.load_checkpoint(image)
    after = b.get_states()
    assert np.array_equal(before["x"], after["x"])  # nothing changed
    with pytest.raises(labf.LabfError):
        a.load_checkpoint(image[:100])
    a.close()
    b.close()


def test_state_calls_restore_the_dynamics_with_step_counters():
    """la_set_states with the step counters (the Philox counters) plus
    la_abf_import of the accumulators restore the dynamics: an engine set
    from another's state continues exactly as that engine does after being
    set from its own state (both rebuild their lists from the same
    positions)."""
    sp, run, st = _inputs()
    a = _engine(sp, run, st)
    a.step(7)
    s = a.get_states()
    assert list(np.asarray(s["step"])) == [7] * 4
    bins = [a.read_abf(0, k) for k in range(len(run.stages))]
    b = _engine(sp, run, st)
    b.set_state(2, step=123)
    assert int(b.get_state(2)["step"]) == 123
    for eng in (a, b):
        eng.set_states(x=np.ascontiguousarray(s["x"]), v=np.ascontiguousarray(s["v"]), lam=s["lam"],
                       plam=s["plam"], step=s["step"])
    for k, r in enumerate(bins):
        b.abf_import(r["sum"], r["sumsq"], r["count"], stage=k)
    assert list(np.asarray(b.get_states()["step"])) == [7] * 4
    a.step(5)
    b.step(5)
    _assert_same(_snapshot(a, run), _snapshot(b, run))
    a.close()
    b.close()


def test_measured_fp_peaks_are_plausible():
    """la_fp_peak: the FP32 FMA rate lies between half and 1.05 x the nominal
    N_SM x 128 lanes x 2 flop x max SM clock; FP64 is far below FP32."""
    import torch

    props = torch.cuda.get_device_properties(0)
    fp32 = labf.fp_peak(False, 0.2)
    fp64 = labf.fp_peak(True, 0.1)
    nominal = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    assert 0.5 * nominal < fp32 < 1.05 * nominal, (fp32, nominal)
    assert 0 < fp64 < 0.25 * fp32
