"""Full-size parity of the neighbour lists: the engine's pair sets
(la_get_pairs) against the oracle's integer pair-set definition (D < R on
quantized coordinates, i < j, exclusions, at most one alchemical atom),
compared exactly, on the bench's own solvation workload (12 300 atoms, list
skin 0.15 nm, 16 walkers), on the largest box of the uneven batch (8192
waters + 40-site solute, 24 616 atoms) and on the 96 040-atom complex
(sampled rows: every pair touching 2000 random atoms and the ligand).  Each
is checked on the lists built from the starting structure and on lists
rebuilt after dynamics (the state is set back, so the lists are built from
exactly the positions the oracle sees).  Many columns, k-d splits, list
capacities and compaction across many super-clusters are exercised here.
"""
import numpy as np
import pytest

import oracle
from paper_2307_08006_gb300 import labf, synth

pytestmark = pytest.mark.gpu


def _relist_and_compare(eng, inputs, walkers, steps, rows=None):
    """Pair sets of `walkers` now, then after `steps` MD steps and a reset of
    every walker to its own state (lists rebuilt from those positions)."""
    def compare(xs):
        row0 = np.concatenate([[0], np.cumsum([si.spec.n * si.run.n_walkers for si in inputs])])
        for w in walkers:
            si_k = eng.walker_sys[w]
            spec = inputs[si_k].spec
            r_list = spec.r_cut + inputs[si_k].run.skin
            x = xs[w]
            pairs, kind = eng.get_pairs(w)
            osys = oracle.OracleSystem(spec)
            if rows is None:
                op, ok = oracle.pair_set(osys, x, r_list)
            else:
                op, ok = oracle.pair_set_rows(osys, x, r_list, rows)
                sel = np.zeros(spec.n, bool)
                sel[rows] = True
                keep = sel[pairs[:, 0]] | sel[pairs[:, 1]]
                pairs, kind = pairs[keep], kind[keep]
            assert len(pairs) > 0
            assert np.array_equal(pairs, op), (w, len(pairs), len(op))
            assert np.array_equal(kind, ok), w

    def per_walker(s):
        out, r = [], 0
        for w in range(eng.n_walkers):
            n = inputs[eng.walker_sys[w]].spec.n
            out.append(np.ascontiguousarray(s["x"][r:r + n]))
            r += n
        return out

    compare(per_walker(eng.get_states()))
    eng.step(steps)
    s = eng.get_states()
    eng.set_states(x=np.ascontiguousarray(s["x"]))
    compare(per_walker(s))


def test_pair_sets_bit_exact_on_the_bench_workload():
    import bench

    spec, run = bench.workload()
    inputs = [labf.SystemInput(spec, run, synth.initial_state(spec, run))]
    eng = labf.Engine(inputs, options=dict(prune_margin=bench.PRUNE_NM))
    assert eng.n_walkers == 16 and spec.n == 12300
    _relist_and_compare(eng, inputs, walkers=(0, 15), steps=200)
    eng.close()


def test_pair_sets_bit_exact_on_the_largest_uneven_box():
    sp = synth.uneven_batch(8008)[-1]
    rng = np.random.default_rng(8015)
    sp.x = ((sp.x + rng.normal(0.0, 0.01, sp.x.shape)) % sp.box).astype(np.float32)
    assert sp.n == 24616
    run = synth.uneven_run(seed=8015, walkers_per_system=2)
    inputs = [labf.SystemInput(sp, run, synth.initial_state(sp, run))]
    eng = labf.Engine(inputs)
    _relist_and_compare(eng, inputs, walkers=(0, 1), steps=100)
    eng.close()


def test_pair_sets_bit_exact_on_the_large_complex_sampled_rows():
    sp = synth.large_complex()
    run = synth.large_complex_run(walkers_per_stage=1)
    inputs = [labf.SystemInput(sp, run, synth.initial_state(sp, run))]
    eng = labf.Engine(inputs)
    rng = np.random.default_rng(8016)
    rows = np.union1d(rng.choice(sp.n, 2000, replace=False), np.nonzero(sp.alch)[0])
    _relist_and_compare(eng, inputs, walkers=(0, 1), steps=20, rows=rows)
    eng.close()
