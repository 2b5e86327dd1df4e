"""Checkpointed correlator runs that resume after a failure.

A production run computes many independent units -- one (configuration,
source) pair each, the correlator C(t) of every nucleus for that pair -- and
a rank can stop half-way (an exception, a killed process, a rank that never
joins).  Each rank keeps an append-only record of the units it has finished:
one JSON line per unit, {"unit": [...], "result": ...}, written with a single
write() after the unit's result exists on the host, then flushed and fsync'd.
On a restart the rank reads its record, skips the recorded units and computes
only the rest; a line torn by a crash (no newline, or not JSON) is ignored, so
that unit is simply computed again.  Units are sharded over ranks with
`sharding.shard` (no data-path collective); `merge` reads every rank's record.

The per-unit computation is the caller's (for the library: build the blocks
of a configuration and contract every table, see `wick_unit`); this module
holds only the bookkeeping and runs on the host.
"""
from __future__ import annotations

import json
import os

from . import sharding


def record_path(base: str, rank: int) -> str:
    return f"{base}.rank{rank}"


def _key(unit) -> str:
    return json.dumps(list(unit))


def read_record(path: str) -> dict:
    """Completed units of one record file: {unit key: result}.  Torn or unreadable lines are skipped."""
    done = {}
    if not os.path.exists(path):
        return done
    with open(path, "rb") as f:
        data = f.read()
    for line in data.split(b"\n")[:-1]:      # the part after the last newline is an unfinished write
        try:
            rec = json.loads(line)
            done[_key(rec["unit"])] = rec["result"]
        except (ValueError, KeyError, TypeError):
            continue
    return done


def _append(path: str, unit, result) -> None:
    line = (json.dumps({"unit": list(unit), "result": result}) + "\n").encode()
    fd = os.open(path, os.O_WRONLY | os.O_CREAT | os.O_APPEND, 0o644)
    try:
        os.write(fd, line)
        os.fsync(fd)
    finally:
        os.close(fd)


def run_units(units, compute, base: str, rank: int = 0, world: int = 1, on_unit=None) -> dict:
    """Compute this rank's share of `units` (a list of tuples, the same list on every rank) that its
    record does not hold yet; compute(unit) returns a JSON-serialisable result.  Returns
    {"computed": [...], "skipped": [...], "results": {unit key: result}} for this rank's share.
    on_unit(unit), if given, is called after each unit is recorded (progress, or a test's failure)."""
    path = record_path(base, rank)
    done = read_record(path)
    mine = [tuple(units[i]) for i in sharding.shard(len(units), rank, world)]
    computed, skipped = [], []
    for u in mine:
        k = _key(u)
        if k in done:
            skipped.append(u)
            continue
        res = compute(u)
        _append(path, u, res)
        done[k] = res
        computed.append(u)
        if on_unit is not None:
            on_unit(u)
    return {"computed": computed, "skipped": skipped, "results": {_key(u): done[_key(u)] for u in mine}}


def merge(base: str, world: int) -> dict:
    """Every rank's completed units: {unit key: result}."""
    out = {}
    for r in range(world):
        out.update(read_record(record_path(base, r)))
    return out


def complex_list(C) -> list:
    """A complex array (any shape) as nested [re, im] pairs, exactly (float64 round-trips through JSON)."""
    import numpy as np
    a = np.asarray(C, dtype=np.complex128)
    return [[float(z.real), float(z.imag)] for z in a.reshape(-1)]


def wick_unit(tables, terms_list, L: int, T: int, precision: int, seed_base: int, dtype=None):
    """compute(unit) for units (configuration, source): synthetic propagators of that configuration's seed
    (sharding.config_seed) and source on the device, the blocks, and C(t) of every table, as
    complex_list of [table][t]."""
    import torch

    from . import wick

    def compute(unit):
        cfg, src = unit
        seed = sharding.config_seed(seed_base, cfg)
        cdt = torch.complex128 if dtype is None else dtype
        Su = torch.empty((1, T, L ** 3, 12, 12), dtype=cdt, device="cuda")
        Sd = torch.empty_like(Su)
        # the source index selects the stream of the generator: source s of a configuration
        wick.wick_synth_propagator(seed, wick.WICK_U, src, L, T, Su)
        wick.wick_synth_propagator(seed, wick.WICK_D, src, L, T, Sd)
        B = torch.empty((1, T, tables.nuc.n_blk), dtype=torch.complex128, device="cuda")
        wick.wick_build_blocks(Su, Sd, tables, precision, B, L, T, 1)
        C = torch.empty((len(terms_list), 1, T), dtype=torch.complex128, device="cuda")
        for i, terms in enumerate(terms_list):
            wick.wick_contract(B, 1, T, terms, precision, C[i])
        return complex_list(C.cpu().numpy())

    return compute
