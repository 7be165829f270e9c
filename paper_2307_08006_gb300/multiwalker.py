"""Multiple walkers spread over several engines (Sec. 2.4).

Walkers of one stage share a single accumulator of the dU/dlambda bin
statistics; each walker biases with the shared statistics plus its own
samples since the last merge.  Inside one engine the device merges every
``shared_freq`` steps.  When the walkers of a stage live in several engines
(one per GPU or process), the systems are created with ``shared_freq = 0``
and the hosts merge instead: every ``exchange_every`` steps each rank
exports its unmerged statistics, all ranks all-gather them, sum them in
rank order (so every rank adds bit-identical totals and the shared
accumulators stay identical) and import the totals.

The exchange moves ``3 * n_bins`` numbers per stage and rank, so it goes
over a CPU (gloo) process group even when the engines run on GPUs.  A rank
that leaves (exception, exit, never joins) makes the others' next exchange
fail with :class:`ExchangeError` once the group's timeout expires or the
peer's connection closes; no exchange is ever left half-applied on a rank,
because the import happens only after every rank's statistics arrived.
"""
from __future__ import annotations

from typing import Iterable, Optional, Sequence, Tuple

import numpy as np


class ExchangeError(RuntimeError):
    """A peer failed or left during a statistics exchange."""


def _dist():
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        raise RuntimeError("torch.distributed is not initialised")
    return torch, dist


def _device_for(dist, group):
    return "cuda" if dist.get_backend(group) == "nccl" else "cpu"


def host_stages(engine) -> Iterable[Tuple[int, int]]:
    """(system, stage) pairs whose merging is left to the host (shared_freq 0)."""
    for si, sysin in enumerate(engine.systems):
        if int(sysin.run.shared_freq) == 0:
            for k in range(len(sysin.run.stages)):
                yield si, k


def check_seeds(engine, group=None) -> None:
    """Raise unless every rank's systems use seeds no other rank uses.

    The Philox key of a walker is (seed, walker index within the engine), so
    two ranks with the same seed would drive their walkers with identical
    noise."""
    torch, dist = _dist()
    seeds = torch.tensor([int(s.run.seed) & 0xFFFFFFFF for s in engine.systems], dtype=torch.int64,
                         device=_device_for(dist, group))
    ws = dist.get_world_size(group)
    got = [torch.empty_like(seeds) for _ in range(ws)]
    try:
        dist.all_gather(got, seeds, group=group)
    except Exception as e:  # noqa: BLE001 - re-raised with context
        raise ExchangeError(f"seed check failed: {e}") from e
    flat = torch.cat(got).tolist()
    if len(set(flat)) != len(flat):
        raise ValueError(f"ranks share Philox seeds {flat}: walkers would see identical noise")


def reduce_in_rank_order(parts: Sequence[np.ndarray]) -> np.ndarray:
    """Sum of per-rank arrays in rank order (the same bits on every rank)."""
    tot = np.array(parts[0], copy=True)
    for p in parts[1:]:
        tot += p
    return tot


def exchange(engine, sys: int, stage: int, group=None) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """One host merge of a stage's statistics across all ranks of ``group``.

    Returns the totals that were imported (identical on every rank)."""
    torch, dist = _dist()
    s1, s2, cnt = engine.abf_export(sys, stage)
    nb = s1.shape[0]
    dev = _device_for(dist, group)
    f = torch.from_numpy(np.concatenate([s1, s2])).to(dev)
    c = torch.from_numpy(cnt).to(dev)
    ws = dist.get_world_size(group)
    fl = [torch.empty_like(f) for _ in range(ws)]
    cl = [torch.empty_like(c) for _ in range(ws)]
    try:
        dist.all_gather(fl, f, group=group)
        dist.all_gather(cl, c, group=group)
    except Exception as e:  # noqa: BLE001 - re-raised with context
        raise ExchangeError(f"exchange of system {sys} stage {stage} failed: {e}") from e
    ftot = reduce_in_rank_order([t.cpu().numpy() for t in fl])
    ctot = reduce_in_rank_order([t.cpu().numpy() for t in cl])
    engine.abf_import(ftot[:nb], ftot[nb:], ctot, sys=sys, stage=stage)
    return ftot[:nb], ftot[nb:], ctot


def run(engine, n_steps: int, exchange_every: int, group=None, check: bool = True) -> int:
    """Advance ``n_steps`` MD steps, merging every ``exchange_every`` steps.

    Every rank must call this with the same ``n_steps`` and
    ``exchange_every``.  Returns the number of exchanges made."""
    if exchange_every <= 0:
        raise ValueError("exchange_every must be positive")
    if check:
        check_seeds(engine, group)
    stages = list(host_stages(engine))
    done, n_ex = 0, 0
    while done < n_steps:
        k = min(exchange_every, n_steps - done)
        engine.step(k)
        done += k
        if k == exchange_every:
            for si, st in stages:
                exchange(engine, si, st, group)
            n_ex += 1
    return n_ex
