"""Resume after a failure (host side, no GPU): the record of completed (configuration, source) units.

The failures are made on the host: a compute that raises after some units, a record line torn by a
crash in mid-write, and a gloo rank that raises between units while the other rank finishes and then
meets the dead rank at the closing barrier (a short process-group timeout ends that wait with an
error).  A restart computes only the units the records do not hold, and the merged results equal an
uninterrupted run's.
"""
import os

import pytest
import torch.multiprocessing as mp

from paper_2411_08962_gb300 import runner

UNITS = [(cfg, src) for cfg in range(5) for src in range(2)]


def fake_compute(unit):
    cfg, src = unit
    return [[cfg * 0.5 + src, -1.0 / (cfg + 1)], [float(src), 3.0]]


class Boom(RuntimeError):
    pass


def test_resume_after_an_exception(tmp_path):
    base = str(tmp_path / "rec")
    calls = []

    def compute(u):
        calls.append(u)
        return fake_compute(u)

    def fail_after_4(u):
        if len(calls) == 4:
            raise Boom(u)

    with pytest.raises(Boom):
        runner.run_units(UNITS, compute, base, on_unit=fail_after_4)
    assert calls == UNITS[:4]
    calls.clear()
    out = runner.run_units(UNITS, compute, base)
    assert calls == UNITS[4:]                         # only the units the record lacks
    assert out["skipped"] == UNITS[:4] and out["computed"] == UNITS[4:]
    clean = runner.run_units(UNITS, fake_compute, str(tmp_path / "clean"))
    assert out["results"] == clean["results"]
    calls.clear()
    again = runner.run_units(UNITS, compute, base)    # everything recorded: nothing recomputed
    assert calls == [] and again["results"] == clean["results"]


def test_torn_record_line_is_recomputed(tmp_path):
    base = str(tmp_path / "rec")
    runner.run_units(UNITS[:3], fake_compute, base)
    path = runner.record_path(base, 0)
    with open(path, "ab") as f:                       # a crash in the middle of the next write
        f.write(b'{"unit": [1, 1], "result": [[1.0, ')
    assert len(runner.read_record(path)) == 3
    calls = []
    out = runner.run_units(UNITS[:4], lambda u: calls.append(u) or fake_compute(u), base)
    assert calls == [UNITS[3]]
    assert out["results"][runner._key(UNITS[3])] == fake_compute(UNITS[3])


def test_results_round_trip_exactly():
    import numpy as np
    C = np.array([1 / 3 + 2j / 7, -1e-300 + 1e300j, 0.1 - 0.2j])
    back = np.array([complex(a, b) for a, b in runner.complex_list(C)])
    assert np.array_equal(back, C)


def _rank(rank, world, port, base, fail_rank, q):
    import datetime

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    done = []

    def fail(u):
        done.append(u)
        if rank == fail_rank and len(done) == 2:
            raise Boom(u)

    try:
        out = runner.run_units(UNITS, fake_compute, base, rank, world, on_unit=fail)
        dist.barrier()                                # a dead peer: error or timeout, not a hang
        q.put((rank, "ok", out["computed"], out["skipped"]))
    except Exception as e:                            # noqa: BLE001 -- reported to the parent
        q.put((rank, type(e).__name__, done, []))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:                             # noqa: BLE001
            pass


def _launch(base, fail_rank, port):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, base, fail_rank, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, status, computed, skipped = q.get(timeout=120)
        res[r] = (status, computed, skipped)
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return res


def test_two_ranks_resume_after_one_fails(tmp_path):
    base = str(tmp_path / "rec")
    port = 29600 + os.getpid() % 1000
    first = _launch(base, fail_rank=1, port=port)
    assert first[1][0] == "Boom"                      # rank 1 failed after its second unit
    assert first[0][0] != "ok" or first[0][1] == UNITS[:5]
    second = _launch(base, fail_rank=-1, port=port + 1)
    assert second[0][0] == "ok" and second[1][0] == "ok"
    assert second[0][1] == [] and second[0][2] == UNITS[:5]          # rank 0 had finished
    assert second[1][2] == UNITS[5:7] and second[1][1] == UNITS[7:]  # rank 1 resumes at its third unit
    merged = runner.merge(base, 2)
    assert merged == {runner._key(u): fake_compute(u) for u in UNITS}
