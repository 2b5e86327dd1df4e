"""Autotuner of the launch tuning (`wick_tuning` of include/wick.h) for a batched workload.

The tunable choices are the block build's range of sites per CTA (the tensor-core
kernel: more sites per CTA mean fewer partial sums and grid-exponent scans, fewer
CTAs to fill the GPU, and coarser fixed-point grids), the contraction's terms per
work item, its CTA size and its resident CTAs per SM.  `tune_batch` times
candidates of the batched executor (`wick.Batch`, created with the candidate in
effect, `run` timed with CUDA events) on the caller's own inputs, one choice at a
time starting from the defaults (coordinate descent), keeps a candidate only if its
correlators agree with the default tuning's within `tol` (the range size moves the
rounding of the block build, the chunking the order of the FP64 term sums), and
returns the choice with every trial -- a JSON-ready dict (`save` writes it, `apply`
sets it process-wide).
"""
from __future__ import annotations

import json

from . import wick

#: candidate values per choice, in the order they are tuned; 0 = the library's default
SPACE = {
    "range_sites": (256, 512, 1024),
    "contract_chunk_terms": (1024, 2048, 4096, 8192, 16384),
    "contract_threads": (128, 256, 512),
    "contract_ctas_per_sm": (0, 2, 4),
}


def _time_batch(batch, stream, reps: int, warmup: int) -> float:
    import torch
    for _ in range(warmup):
        batch.run(stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        batch.run(stream)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune_batch(Su_list, Sd_list, tables, terms_list, precision, L, T, n_src, reps: int = 3, warmup: int = 1,
               space=None, tol: float = 1e-9, stream=None) -> dict:
    """Coordinate-descent search over `space` (default SPACE) for the batch of the given inputs.
    Returns {"choice": tuning dict, "ms_per_run": best time, "default_ms_per_run": time with the
    defaults, "trials": [...]}; the process-wide tuning is left as it was."""
    import torch
    space = SPACE if space is None else space
    stream = torch.cuda.current_stream() if stream is None else stream
    saved = wick.wick_get_tuning()
    n = len(Su_list)
    blocks = torch.empty((n, n_src, T, tables.nuc.n_blk), dtype=torch.complex128, device="cuda")
    C = torch.empty((n, len(terms_list), n_src, T), dtype=torch.complex128, device="cuda")
    trials, ref = [], None

    def measure(tuning):
        nonlocal ref
        wick.wick_set_tuning(tuning)
        batch = wick.Batch(Su_list, Sd_list, tables, terms_list, precision, blocks, C, L, T, n_src)
        try:
            ms = _time_batch(batch, stream, reps, warmup)
        finally:
            batch.free()
        got = C.clone()
        if ref is None:
            ref = got
        diff = float(((got - ref).abs() / ref.abs()).max().item())
        rec = {"tuning": dict(tuning), "ms_per_run": ms, "max_rel_diff_vs_default": diff, "accepted": diff <= tol}
        trials.append(rec)
        return rec

    try:
        best = {f: 0 for f in wick.TUNING_FIELDS}
        base = measure(best)
        best_ms = base["ms_per_run"]
        for field, values in space.items():
            for v in values:
                if v == best[field]:
                    continue
                cand = dict(best, **{field: v})
                rec = measure(cand)
                if rec["accepted"] and rec["ms_per_run"] < best_ms:
                    best, best_ms = cand, rec["ms_per_run"]
    finally:
        wick.wick_set_tuning(saved)
    return {"choice": best, "ms_per_run": best_ms, "default_ms_per_run": base["ms_per_run"], "configs": n,
            "reps": reps, "tol": tol, "trials": trials}


def save(result: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump(result, f, indent=1)


def load(path: str) -> dict:
    with open(path) as f:
        return json.load(f)


def apply(result: dict) -> None:
    """Make a tuner result's choice the process-wide tuning."""
    wick.wick_set_tuning(result["choice"])
