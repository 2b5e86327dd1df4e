"""Host-side checks of the C ABI and the product's operator tables (no GPU).

* libwick.so builds, loads and exports every function include/wick.h declares;
* the host-only entry points work without a device (block counts, error
  strings, file validation);
* the product's operator/nucleus tables equal the oracle's, built by separate
  code from the same definitions, so both sides enumerate the same raw terms.
"""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import operators as oops
from paper_2411_08962_gb300 import build, operators, wick

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wick.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return wick.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*[\s\*]+(wick_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_binding_exports():
    assert set(declared_functions()) == set(wick.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", wick.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s[TW]\s(wick_[a-z_0-9]+)$", out, flags=re.M))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_host_only_calls(lib):
    assert wick.wick_version() == "0.1.0"
    assert wick.strerror(wick.WICK_EIO).startswith("term-table file")
    nuc = operators.nucleus("he4")
    t = wick.Tables(nuc)
    assert wick.wick_block_count(t) == 2 * 2 * 6 ** 3 == nuc.n_blk
    bad = wick.wick_block_layout(2, 2, 3, (C.c_int8 * 12)(0, 0, 1))   # not ascending
    assert lib.wick_block_count(C.byref(bad)) == 0


def test_terms_file_validation(lib, tmp_path):
    h = C.c_void_p(None)
    assert lib.wick_terms_load(str(tmp_path / "missing.bin").encode(), C.byref(h)) == wick.WICK_EIO
    p = tmp_path / "junk.bin"
    p.write_bytes(b"WICKTBL1" + os.urandom(64))
    assert lib.wick_terms_load(str(p).encode(), C.byref(h)) == wick.WICK_EIO
    assert not h.value


def test_null_arguments_are_rejected(lib):
    h = C.c_void_p(None)
    assert lib.wick_reduce_terms(None, None, None, 0, 2, 1, C.byref(h), None) == wick.WICK_EINVAL
    assert lib.wick_build_blocks(None, None, None, None, 0, None, None) == wick.WICK_EINVAL
    assert lib.wick_contract(None, 1, 1, None, 0, None, None) == wick.WICK_EINVAL
    n = C.c_size_t(0)
    assert lib.wick_upload_rows(None, None, None, None, None, None, wick.WICK_UPLOAD_AUTO, C.byref(n),
                                None) == wick.WICK_EINVAL
    assert lib.wick_det_contract(None, None, None, 1.0, wick.WICK_FP64, None, None) == wick.WICK_EINVAL


def test_upload_rows_rejects_bad_mode_and_host_memory(lib):
    """Argument checks that run before any device work: an unknown mode, and host memory that is not
    page-locked (no CUDA device here, so no host buffer can be)."""
    tabs = wick.Tables(operators.nucleus("he4"))
    host = np.zeros(2 * 1 * 8 * 144, dtype=np.complex64)
    dev = np.zeros(2 * 1 * 8 * 144 + 2, dtype=np.complex64)   # stands in for a device pointer: only checked
    dptr = dev.ctypes.data + (-dev.ctypes.data) % 16           # for 16-byte alignment before the mode / host
    hp = wick.wick_prop(host.ctypes.data, 2, 1, 1, wick.WICK_C64)
    dp = wick.wick_prop(dptr, 2, 1, 1, wick.WICK_C64)
    n = C.c_size_t(0)
    for mode in (7, -1):
        assert lib.wick_upload_rows(C.byref(hp), C.byref(hp), C.byref(dp), C.byref(dp), tabs.ops,
                                    C.byref(tabs.layout), mode, C.byref(n), None) == wick.WICK_EINVAL
    assert lib.wick_upload_rows(C.byref(hp), C.byref(hp), C.byref(dp), C.byref(dp), tabs.ops,
                                C.byref(tabs.layout), wick.WICK_UPLOAD_DMA, C.byref(n), None) == wick.WICK_EINVAL
    assert n.value == 0


def test_product_dirac_algebra():
    g = operators.dirac_matrices()
    for mu in range(4):
        for nu in range(4):
            assert np.allclose(g[mu] @ g[nu] + g[nu] @ g[mu], 2 * (mu == nu) * np.eye(4))
    G = operators.diquark_matrix()
    assert np.array_equal(G, -G.T) and np.array_equal(G, oops.integer_matrix(oops.cg5()))
    assert np.array_equal(operators.diquark_matrix(+1)[:2, :2], G[:2, :2])


@pytest.mark.parametrize("name", ["proton", "deuteron", "he3", "he4"])
@pytest.mark.parametrize("form", ["upper", "full"])
def test_product_tables_equal_oracle_tables(name, form):
    if name in ("he3", "he4") and form == "full":
        pytest.skip("full-spin He-3/He-4 source tables are large; the nucleon tables are compared below")
    a = operators.nucleus(name, form)
    b = oops.nucleus(name, form)
    assert a.A == b["A"] and a.n_spin == b["n_spin"] and list(a.chi) == list(b["chi"])
    for (f, tab), op in zip(b["ops"], a.ops):
        assert f == op.flav_pair and [tuple(e) for e in tab] == [tuple(e) for e in op.entries]
    assert [tuple(s) for s in a.sink] == [tuple(s) for s in b["sink"]]
    assert a.src == b["src"]
    assert list(a.src_flav) == list(b["src_flav"])
    assert a.n_raw == oops.n_raw_terms(b)


def test_binding_rejects_bad_tensors_before_the_library(lib):
    """The C side cannot see the size, dtype or placement of a buffer; the binding checks them and
    raises ValueError before anything reaches libwick (a bad buffer would otherwise be read or
    written out of bounds on the device)."""
    import types

    torch = pytest.importorskip("torch")
    tabs = wick.Tables(operators.nucleus("deuteron"))
    L, T, n_src = 2, 2, 1
    n_prop = n_src * T * L ** 3 * 144
    nb = tabs.nuc.n_blk
    good_s = torch.zeros(n_prop, dtype=torch.complex64)
    good_b = torch.zeros(n_src * T * nb, dtype=torch.complex128)
    cases = {
        "wrong propagator dtype": (torch.zeros(n_prop, dtype=torch.float64), good_b),
        "non-contiguous propagator": (torch.zeros(2 * n_prop, dtype=torch.complex64)[::2], good_b),
        "short propagator": (torch.zeros(n_prop - 1, dtype=torch.complex64), good_b),
        "host propagator": (good_s, good_b),
        "complex64 blocks": (good_s, torch.zeros(n_src * T * nb, dtype=torch.complex64)),
        "short blocks": (good_s, torch.zeros(n_src * T * nb - 1, dtype=torch.complex128)),
    }
    for what, (S, B) in cases.items():
        with pytest.raises(ValueError):
            wick.wick_build_blocks(S, S, tabs, wick.WICK_FP64, B, L, T, n_src)
    fake_terms = types.SimpleNamespace(block_count=nb, h=None)
    with pytest.raises(ValueError):   # output too small
        wick.wick_contract(good_b, n_src, T, fake_terms, wick.WICK_FP64,
                           torch.zeros(n_src * T - 1, dtype=torch.complex128))
    with pytest.raises(ValueError):   # blocks of another layout (too few entries per slice)
        wick.wick_contract_noalloc(torch.zeros(n_src * T * (nb - 1), dtype=torch.complex128), n_src, T,
                                   fake_terms, wick.WICK_FP64, torch.zeros(n_src * T, dtype=torch.complex128))
    with pytest.raises(ValueError):   # host tensors
        wick.wick_contract(good_b, n_src, T, fake_terms, wick.WICK_FP64, torch.zeros(n_src * T, dtype=torch.complex128))
    with pytest.raises(ValueError):   # upload source not page-locked
        wick.wick_upload_rows(good_s, good_s, good_s, good_s, tabs, L, T, n_src)
    with pytest.raises(ValueError):
        wick.wick_cluster_product(torch.zeros(4, dtype=torch.complex128), torch.zeros(3, dtype=torch.complex128),
                                  torch.zeros(4, dtype=torch.complex128))
    with pytest.raises(ValueError):
        wick.wick_synth_propagator(1, 0, 0, L, T, torch.zeros(n_prop // n_src - 1, dtype=torch.complex64))


def test_tuning_is_validated_and_kept(lib):
    """wick_set_tuning checks every field and is read back by wick_get_tuning (host-only calls)."""
    try:
        wick.wick_set_tuning({"range_sites": 1024, "contract_threads": 128, "contract_chunk_terms": 2048})
        assert wick.wick_get_tuning() == {"range_sites": 1024, "contract_threads": 128, "contract_ctas_per_sm": 0,
                                          "contract_chunk_terms": 2048, "hash_log2_start": 0, "hash_log2_max": 0,
                                          "no_pair_kernel": 0}
        for bad in ({"range_sites": 100}, {"range_sites": 8192}, {"contract_threads": 100},
                    {"contract_threads": 1024}, {"contract_ctas_per_sm": -1}, {"contract_chunk_terms": 10},
                    {"hash_log2_start": 3}, {"hash_log2_start": 29}, {"hash_log2_max": 2}, {"hash_log2_max": 30},
                    {"no_pair_kernel": 2}):
            with pytest.raises(wick.WickError) as e:
                wick.wick_set_tuning(bad)
            assert e.value.code == wick.WICK_EINVAL
        assert wick.wick_get_tuning()["range_sites"] == 1024      # a refused tuning changes nothing
    finally:
        wick.wick_set_tuning(None)
    assert wick.wick_get_tuning() == {f: 0 for f in wick.TUNING_FIELDS}


def test_autotune_choice_round_trips(lib, tmp_path):
    """A tuner result saved as JSON loads back and applies as the process-wide tuning (host only)."""
    from paper_2411_08962_gb300 import autotune
    res = {"choice": dict({f: 0 for f in wick.TUNING_FIELDS}, range_sites=2048, contract_chunk_terms=16384),
           "ms_per_run": 1.0, "default_ms_per_run": 1.1, "trials": []}
    path = str(tmp_path / "tuning.json")
    autotune.save(res, path)
    back = autotune.load(path)
    assert back == res
    try:
        autotune.apply(back)
        assert wick.wick_get_tuning() == back["choice"]
    finally:
        wick.wick_set_tuning(None)
    assert wick.wick_get_tuning() == {f: 0 for f in wick.TUNING_FIELDS}


def test_selftest_wait_checks_its_arguments(lib):
    """The bounded-wait self-test refuses an unknown wait or a limit outside 1 .. 2^22 before touching
    the device."""
    for which, limit in ((2, 100), (-1, 100), (0, 0), (1, (1 << 22) + 1)):
        with pytest.raises(wick.WickError) as e:
            wick.wick_selftest_wait(which, limit)
        assert e.value.code == wick.WICK_EINVAL


def test_alloc_failure_injection_is_host_state():
    """The injection is a process-wide countdown on the host: set, read back, cancelled (no GPU call)."""
    assert wick.wick_inject_alloc_failure(0) == 0
    assert wick.wick_inject_alloc_failure(3) == 0
    assert wick.wick_inject_alloc_failure(5) == 3      # nothing allocated since: still 3 to go
    assert wick.wick_inject_alloc_failure(0) == 5
    with pytest.raises(wick.WickError) as e:
        wick.wick_inject_alloc_failure(-1)
    assert e.value.code == wick.WICK_EINVAL


def test_product_planewave_operators_equal_oracle():
    """The correlation-matrix basis and the plane-wave NP operator: the product's tables equal the
    oracle's, built by separate code from the same definitions."""
    pairs = list(zip(operators.deuteron_pw_basis(), oops.deuteron_pw_basis()))
    pairs.append((operators.deuteron_np(), oops.deuteron_np_planewave()))
    for a, b in pairs:
        assert a.A == b["A"] and a.n_spin == b["n_spin"] and list(a.chi) == list(b["chi"])
        for (f, tab), op in zip(b["ops"], a.ops):
            assert f == op.flav_pair and [tuple(e) for e in tab] == [tuple(e) for e in op.entries]
        assert [tuple(s) for s in a.sink] == [tuple(s) for s in b["sink"]]
        assert a.src == b["src"] and list(a.src_flav) == list(b["src_flav"])


@pytest.mark.parametrize("name", ["deuteron", "he3", "he4"])
def test_nucleon_tables_are_symmetric_under_diquark_exchange(name):
    """The tensor-core build shares one computation of the diquark values between the proton and the
    neutron type (their values are each other's with the columns transposed) only when each table is
    unchanged by exchanging the two diquark slots: swapping the colours of the epsilon and the spins of
    the antisymmetric C gamma5 flips two signs.  Pinned on the product's tables for the upper-spin
    nuclei, and the two types hold the same table with opposite pair flavours."""
    nuc = operators.nucleus(name)
    assert len(nuc.ops) == 2 and {op.flav_pair for op in nuc.ops} == {0, 1}
    assert nuc.ops[0].entries == nuc.ops[1].entries
    for op in nuc.ops:
        entries = {tuple(e) for e in op.entries}
        swapped = {(s, q1, q3, q2, w) for s, q1, q2, q3, w in op.entries}
        assert entries == swapped
