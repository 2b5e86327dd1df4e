"""Failure detection on the GPU, driven from the host: no test faults, traps or hangs a GPU.

* bounded waits: each of the library's device waits (a hash-table slot claimed by another thread, an
  mbarrier phase of the tensor-core block build) is run on a flag that nothing sets with a short poll
  limit; the kernel gives up, records WICK_ETIMEOUT in its status word and returns, and the context
  stays usable (a reduction and a contraction afterwards match the ones before);
* capacity: the reduction's hash table grows by doubling from a tiny first size (same table, bit for
  bit) and, with its largest size capped below what the nucleus needs, fails with WICK_ECAPACITY;
* overflow: a weight product past the in-warp int32 sums, and a stored table whose weight reaches 2^53,
  are refused with WICK_EOVERFLOW before anything runs on the device;
* allocation failures: injected on the host (the library's allocator reports failure without calling
  cudaMalloc) at each allocation point of a call in turn; every such call returns WICK_ENOMEM, frees
  what it took, and the next call succeeds with the same results.
"""
import struct

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2411_08962_gb300 import build, operators, synth, wick  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    wick.load()
    yield
    wick.wick_set_tuning(None)
    wick.wick_inject_alloc_failure(0)


def table(name):
    t = wick.wick_reduce_terms(wick.Tables(operators.nucleus(name)))
    ids, w, rep = t.copy()
    t.free()
    return ids, w, rep


def correlator(tabs, terms, L=4, T=4, n_src=1, seed=11):
    Su = torch.from_numpy(synth.propagator(seed, 0, L, T, n_src)).cuda()
    Sd = torch.from_numpy(synth.propagator(seed, 1, L, T, n_src)).cuda()
    B = torch.empty((n_src, T, tabs.nuc.n_blk), dtype=torch.complex128, device="cuda")
    wick.wick_build_blocks(Su, Sd, tabs, wick.WICK_FP64, B, L, T, n_src)
    C = torch.empty((n_src, T), dtype=torch.complex128, device="cuda")
    wick.wick_contract(B, n_src, T, terms, wick.WICK_FP64, C)
    torch.cuda.synchronize()
    return C.cpu().numpy()


@pytest.mark.parametrize("which", [0, 1], ids=["hash_slot", "mbarrier"])
def test_bounded_wait_runs_out_and_reports(which):
    tabs = wick.Tables(operators.nucleus("deuteron"))
    terms = wick.wick_reduce_terms(tabs)
    before = correlator(tabs, terms)
    assert wick.wick_selftest_wait(which, 1000) == wick.WICK_ETIMEOUT
    assert wick.wick_status() == wick.WICK_OK          # the word was read and cleared
    torch.cuda.synchronize()
    after = correlator(tabs, terms)                     # the context is still usable
    assert np.array_equal(before, after)
    with pytest.raises(wick.WickError):
        wick.wick_selftest_wait(which, 0)               # limits outside 1 .. 2^22 are refused
    with pytest.raises(wick.WickError):
        wick.wick_selftest_wait(2, 10)


def test_hash_table_grows_and_caps():
    ref = table("he3")
    try:
        wick.wick_set_tuning({"hash_log2_start": 4})   # 16 slots: several rounds of doubling
        got = table("he3")
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)
        wick.wick_set_tuning({"hash_log2_start": 4, "hash_log2_max": 6})   # 64 slots: too few
        with pytest.raises(wick.WickError) as e:
            table("he3")
        assert e.value.code == wick.WICK_ECAPACITY
    finally:
        wick.wick_set_tuning(None)
    got = table("he3")
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_weight_overflow_is_refused():
    nuc = operators.nucleus("deuteron")
    nuc.sink = [(t, s, w * (1 << 30)) for t, s, w in nuc.sink]   # 32 x sink x source weight >= 2^31
    with pytest.raises(wick.WickError) as e:
        wick.wick_reduce_terms(wick.Tables(nuc))
    assert e.value.code == wick.WICK_EOVERFLOW


def _fnv1a(data: bytes, h: int) -> int:
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def test_stored_weight_past_2_53_is_refused(tmp_path):
    """A table file whose weight cannot be held exactly by the FP64 contraction: WICK_EOVERFLOW on load."""
    terms = wick.wick_reduce_terms(wick.Tables(operators.nucleus("deuteron")))
    path = str(tmp_path / "d.wtb")
    terms.save(path)
    raw = bytearray(open(path, "rb").read())
    # layout: magic 8, version 4, 5 x int32, chi 12, U 8, scale 8, stats 4 x 8, bound 8, ids, w, rep, hash 8
    U = struct.unpack_from("<q", raw, 8 + 4 + 20 + 12)[0]
    A = struct.unpack_from("<i", raw, 8 + 4)[0]
    head = 8 + 4 + 20 + 12 + 8 + 8 + 32 + 8
    w_off = head + 2 * U * A
    struct.pack_into("<q", raw, w_off, 1 << 60)
    body = bytes(raw[head:head + 2 * U * A + 16 * U])
    h = _fnv1a(body, 1469598103934665603)
    struct.pack_into("<Q", raw, len(raw) - 8, h)
    open(path, "wb").write(bytes(raw))
    with pytest.raises(wick.WickError) as e:
        wick.Terms.load_file(path)
    assert e.value.code == wick.WICK_EOVERFLOW
    # the untouched file still loads
    terms.save(path)
    t2 = wick.Terms.load_file(path)
    assert t2.count == terms.count


def fail_each_allocation(call, max_points=64):
    """Run call() with its k-th device allocation failing, k = 1, 2, ... until it makes fewer than k
    allocations (and succeeds); every failing run must raise WICK_ENOMEM.  Returns the failure points."""
    for k in range(1, max_points + 1):
        wick.wick_inject_alloc_failure(k)
        try:
            call()
        except wick.WickError as e:
            assert e.code == wick.WICK_ENOMEM, e.args[0]
            assert wick.wick_inject_alloc_failure(0) == 0      # the k-th allocation was the one refused
            continue
        assert wick.wick_inject_alloc_failure(0) > 0           # fewer than k allocations: nothing refused
        return k - 1
    raise AssertionError("more allocation points than expected")


def test_injected_allocation_failures(tmp_path):
    ref = table("he3")
    tabs = wick.Tables(operators.nucleus("he3"))
    n_points = fail_each_allocation(lambda: wick.wick_reduce_terms(tabs).free())
    assert n_points >= 3
    got = table("he3")
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    # a batch whose scratch cannot be allocated: refused, nothing left behind; then built and run
    dtabs = wick.Tables(operators.nucleus("deuteron"))
    terms = wick.wick_reduce_terms(dtabs)
    L, T, n_src = 4, 4, 1
    Su = [torch.from_numpy(synth.propagator(3, 0, L, T, n_src)).cuda()]
    Sd = [torch.from_numpy(synth.propagator(3, 1, L, T, n_src)).cuda()]
    B = torch.empty((1, n_src, T, dtabs.nuc.n_blk), dtype=torch.complex128, device="cuda")
    C = torch.empty((1, 1, n_src, T), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert fail_each_allocation(lambda: wick.Batch(Su, Sd, dtabs, [terms], wick.WICK_FP64, B, C, L, T,
                                                   n_src).free()) >= 2
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)   # the failed creates freed what they took
    b = wick.Batch(Su, Sd, dtabs, [terms], wick.WICK_FP64, B, C, L, T, n_src)
    b.run()
    torch.cuda.synchronize()
    assert np.array_equal(C[0, 0].cpu().numpy(), correlator(dtabs, terms, seed=3))
    b.free()
    # a stored table whose device copies cannot be allocated
    path = str(tmp_path / "d.wtb")
    terms.save(path)
    assert fail_each_allocation(lambda: wick.Terms.load_file(path).free()) >= 2


def test_resumed_run_equals_uninterrupted(tmp_path):
    """runner.run_units with the library's per-unit computation (blocks and correlators of one
    (configuration, source) on the device): a run that fails after two units and is restarted computes
    only the missing units, and every unit's C(t) equals an uninterrupted run's bit for bit."""
    from paper_2411_08962_gb300 import runner
    tabs = wick.Tables(operators.nucleus("deuteron"))
    terms = [wick.wick_reduce_terms(tabs)]
    units = [(cfg, src) for cfg in range(3) for src in range(2)]
    compute = runner.wick_unit(tabs, terms, L=4, T=4, precision=wick.WICK_FP64, seed_base=0x51)

    class Stop(RuntimeError):
        pass

    done = []

    def stop_after_two(u):
        done.append(u)
        if len(done) == 2:
            raise Stop()

    base = str(tmp_path / "run")
    with pytest.raises(Stop):
        runner.run_units(units, compute, base, on_unit=stop_after_two)
    out = runner.run_units(units, compute, base)
    assert out["skipped"] == units[:2] and out["computed"] == units[2:]
    clean = runner.run_units(units, compute, str(tmp_path / "clean"))
    assert out["results"] == clean["results"]
    # and each unit is the correlator of its configuration's source
    c = np.array([complex(a, b) for a, b in out["results"][runner._key(units[3])]])
    assert c.shape == (4,) and np.all(np.isfinite(c)) and np.all(c != 0)
