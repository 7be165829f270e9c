"""Host-level multiple-walker exchange (Sec. 2.4) over a world-size-2 gloo
group on the CPU.

The engines are stand-ins that hold the two accumulators the CUDA engine
keeps per stage (shared statistics, unmerged per-walker statistics) and
draw their samples from a seeded generator, so that the protocol (rank
order, identical totals on every rank, clearing, failure of a peer) is
tested without a GPU.  The engine side of export/import is tested on the
GPU against the on-device merge.
"""
import datetime
import os
import socket
import traceback
from types import SimpleNamespace

import numpy as np
import pytest
import torch.multiprocessing as mp

N_BINS = 7


class FakeEngine:
    """Two stages; every step each walker adds one sample to a random bin."""

    def __init__(self, seed, walkers=3, shared_freq=0):
        run = SimpleNamespace(seed=seed, shared_freq=shared_freq,
                              stages=[SimpleNamespace(n_bins=N_BINS), SimpleNamespace(n_bins=N_BINS)])
        self.systems = [SimpleNamespace(run=run)]
        self.rng = np.random.default_rng(seed)
        self.walkers = walkers
        z = lambda: [np.zeros(N_BINS), np.zeros(N_BINS), np.zeros(N_BINS, np.int64)]
        self.shared = [z(), z()]
        self.local = [z(), z()]
        self.samples = [z(), z()]  # every sample ever drawn (for checking)
        self.steps = 0

    def step(self, n):
        for _ in range(n):
            for st in range(2):
                for _w in range(self.walkers):
                    k = int(self.rng.integers(N_BINS))
                    v = float(self.rng.normal(3.0 * st, 1.0))
                    for acc in (self.local[st], self.samples[st]):
                        acc[0][k] += v
                        acc[1][k] += v * v
                        acc[2][k] += 1
        self.steps += n

    def abf_export(self, sys, stage):
        return tuple(a.copy() for a in self.local[stage])

    def abf_import(self, s1, s2, c, sys=0, stage=0):
        for a, b in zip(self.shared[stage], (s1, s2, c)):
            a += b
        self.local[stage] = [np.zeros(N_BINS), np.zeros(N_BINS), np.zeros(N_BINS, np.int64)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _leave(q, msg):
    """Report and exit at once (flushes the queue's feeder thread first)."""
    q.put(msg)
    q.close()
    q.join_thread()
    os._exit(0)


def _worker(rank, world, port, mode, q):
    import torch.distributed as dist

    from paper_2307_08006_gb300 import multiwalker
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=10))
        seed = 100 if mode == "same_seed" else 100 + rank
        eng = FakeEngine(seed, walkers=2 + rank)
        if mode == "dropout" and rank == 1:
            eng.step(5)
            dist.destroy_process_group()
            _leave(q, (rank, "left", None))  # leaves between steps, nothing in flight
        try:
            n_ex = multiwalker.run(eng, 23, 5, check=True)
        except multiwalker.ExchangeError as e:
            _leave(q, (rank, "exchange_error", str(e)))
        except ValueError as e:
            _leave(q, (rank, "value_error", str(e)))
        # every rank's samples, for the check in the parent
        q.put((rank, "ok", dict(n_ex=n_ex, shared=[[a.tolist() for a in s] for s in eng.shared],
                                local=[[a.tolist() for a in s] for s in eng.local],
                                samples=[[a.tolist() for a in s] for s in eng.samples])))
        dist.destroy_process_group()
    except Exception:  # noqa: BLE001 - reported to the parent
        q.put((rank, "crash", traceback.format_exc()))


def _launch(mode, world=2, wait=60):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(world):
            r, kind, payload = q.get(timeout=wait)
            out[r] = (kind, payload)
    finally:
        for p in procs:
            p.join(timeout=10)
            if p.is_alive():
                p.kill()
                p.join()
    return out


def test_exchange_rank_order_totals_identical():
    out = _launch("normal")
    assert {k for k, _ in out.values()} == {"ok"}, out
    r0, r1 = out[0][1], out[1][1]
    assert r0["n_ex"] == r1["n_ex"] == 4  # 23 steps, exchange every 5
    for st in range(2):
        # identical shared statistics on both ranks (bit for bit)
        for a, b in zip(r0["shared"][st], r1["shared"][st]):
            assert a == b
        # shared + still-unmerged local samples account for every sample
        for j in range(3):
            tot = np.asarray(r0["samples"][st][j]) + np.asarray(r1["samples"][st][j])
            have = (np.asarray(r0["shared"][st][j]) + np.asarray(r0["local"][st][j]) +
                    np.asarray(r1["local"][st][j]))
            np.testing.assert_allclose(have, tot, rtol=1e-12, atol=1e-9)
        # counts are exact: 20 merged steps of (2 + 3) walkers
        assert int(np.sum(r0["shared"][st][2])) == 20 * 5
        assert int(np.sum(r0["local"][st][2])) == 3 * 2
        assert int(np.sum(r1["local"][st][2])) == 3 * 3


def test_shared_seed_is_refused():
    out = _launch("same_seed")
    assert [out[r][0] for r in (0, 1)] == ["value_error", "value_error"], out


def test_rank_dropout_fails_the_exchange():
    out = _launch("dropout", wait=90)
    assert out[1][0] == "left"
    assert out[0][0] == "exchange_error", out


def test_reduce_in_rank_order_is_sequential():
    from paper_2307_08006_gb300 import multiwalker
    parts = [np.array([1e16]), np.array([1.0]), np.array([-1e16])]
    # rank order: (1e16 + 1) - 1e16 = 0 in double (1 is below half an ulp of
    # 1e16); any other association, e.g. 1e16 - 1e16 first, gives 1
    assert multiwalker.reduce_in_rank_order(parts)[0] == 0.0
    assert multiwalker.reduce_in_rank_order([parts[0], parts[2], parts[1]])[0] == 1.0
    with pytest.raises(ValueError):
        multiwalker.run(FakeEngine(1), 5, 0)
