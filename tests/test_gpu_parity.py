"""GPU parity: the CUDA path through the C ABI against the CPU reference.

Tolerances (stated by the method's precision contract): reduced term tables
bit-exact; FP64 path <= 1e-12 relative per time slice; mixed path (FP32
products, FP64 sums) <= 1e-6 relative per time slice.  Blocks are compared
entry-wise relative to the largest entry of their slice.
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import operators as oops  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2411_08962_gb300 import build, operators, synth, wick  # noqa: E402

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
import make_tables  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    wick.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_blocks(Su, Sd, tabs, precision):
    nuc = tabs.nuc
    n_src, T, V = Su.shape[:3]
    L = round(V ** (1 / 3))
    out = torch.empty((n_src, T, nuc.n_blk), dtype=torch.complex128, device="cuda")
    wick.wick_build_blocks(dev(Su), dev(Sd), tabs, wick.WICK_MIXED if precision == "mixed" else wick.WICK_FP64,
                           out, L, T, n_src)
    torch.cuda.synchronize()
    return out


def gpu_contract(blocks, terms, precision):
    n_src, T = blocks.shape[:2]
    C = torch.empty((n_src, T), dtype=torch.complex128, device="cuda")
    wick.wick_contract(blocks, n_src, T, terms, wick.WICK_MIXED if precision == "mixed" else wick.WICK_FP64, C)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def rel_per_t(a, b):
    return np.max(np.abs(a - b) / np.abs(b))


def block_err(gpu, ref):
    ref = ref.reshape(gpu.shape)
    scale = np.max(np.abs(ref), axis=-1, keepdims=True)
    return np.max(np.abs(gpu - ref) / scale)


def props(L, T, n_src, seed, dtype=np.complex128):
    return (synth.propagator(seed, 0, L, T, n_src, dtype=dtype), synth.propagator(seed, 1, L, T, n_src, dtype=dtype))


def oracle_blocks(Su, Sd, name, form="upper"):
    onuc = oops.nucleus(name, form)
    return O.antisymmetric_blocks(O.blocks_single(Su.astype(np.complex128), Sd.astype(np.complex128), onuc), onuc)


# ---------------------------------------------------------------------------
# blocks
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("L,T,n_src,form", [
    (4, 8, 1, "upper"),    # the deuteron workload
    (3, 3, 2, "upper"),    # ragged: 27 sites
    (7, 2, 1, "upper"),    # 343 sites: two site chunks with a ragged tail
    (1, 1, 1, "upper"),    # a single site
    (2, 2, 1, "full"),     # all four spins: several output chunks
])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_blocks_match_oracle(L, T, n_src, form, precision):
    Su, Sd = props(L, T, n_src, seed=L * 100 + T)
    tabs = wick.Tables(operators.nucleus("deuteron", form))
    B = gpu_blocks(Su, Sd, tabs, precision).cpu().numpy()
    ref = oracle_blocks(Su, Sd, "deuteron", form)
    tol = FP64_TOL if precision == "fp64" else MIXED_TOL
    assert block_err(B, ref) < tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_blocks_general_integer_weights(precision):
    """Diquark weights that are not powers of two (3 C gamma5) take the scalar
    double-FP32 path of the mixed block kernel."""
    G3 = 3 * operators.diquark_matrix()
    nuc = operators.nucleus("deuteron")
    nuc.ops = [operators.nucleon_op(operators.U, G3, (0, 1), (0, 1)),
               operators.nucleon_op(operators.D, G3, (0, 1), (0, 1))]
    Su, Sd = props(3, 2, 1, seed=17, dtype=np.complex64)
    B = gpu_blocks(Su, Sd, wick.Tables(nuc), precision).cpu().numpy()
    onuc = oops.nucleus("deuteron")
    tab3 = oops.nucleon_table(3 * oops.cg5(), oops.UPPER, oops.UPPER)
    onuc["ops"] = [(oops.U, tab3), (oops.D, tab3)]
    ref = O.antisymmetric_blocks(O.blocks_single(Su.astype(np.complex128), Sd.astype(np.complex128), onuc), onuc)
    assert block_err(B, ref) < (FP64_TOL if precision == "fp64" else MIXED_TOL)


def test_blocks_c64_storage_fp64_arithmetic():
    Su, Sd = props(4, 2, 1, seed=5, dtype=np.complex64)
    tabs = wick.Tables(operators.nucleus("deuteron"))
    B = gpu_blocks(Su, Sd, tabs, "fp64").cpu().numpy()
    assert block_err(B, oracle_blocks(Su, Sd, "deuteron")) < FP64_TOL


def test_blocks_exact_antisymmetry_and_isospin():
    Su, _ = props(4, 2, 1, seed=9)
    tabs = wick.Tables(operators.nucleus("deuteron"))
    B = gpu_blocks(Su, Su, tabs, "fp64").cpu().numpy().reshape(1, 2, 2, 2, 6, 6, 6)
    assert np.array_equal(B, -B.swapaxes(-3, -2))           # Eq. 2.4: odd under chi'1 <-> chi'2
    assert np.array_equal(B[:, :, 0], B[:, :, 1])          # S_u = S_d  =>  B^p = B^n


def test_blocks_deterministic():
    Su, Sd = props(8, 2, 1, seed=3, dtype=np.complex64)
    tabs = wick.Tables(operators.nucleus("deuteron"))
    a = gpu_blocks(Su, Sd, tabs, "mixed")
    b = gpu_blocks(Su, Sd, tabs, "mixed")
    assert torch.equal(a, b)


# ---------------------------------------------------------------------------
# reduced term tables
# ---------------------------------------------------------------------------
def gpu_table(name, seed=0x2411, sites=1, form="upper"):
    tabs = wick.Tables(operators.nucleus(name, form))
    terms = wick.wick_reduce_terms(tabs, seed=seed, sites=sites)
    return terms, terms.copy(), terms.stats()


@pytest.mark.parametrize("name", ["proton", "deuteron", "he3"])
def test_reduced_table_bit_exact(name):
    _, g, (stats, bound) = gpu_table(name)
    o = O.dedup(oops.nucleus(name), seed=77)
    assert np.array_equal(g["rep"], o["rep"])
    assert np.array_equal(g["w"], o["w"])
    assert np.array_equal(g["ids"], o["ids"])
    assert stats == o["stats"]
    assert 0.0 <= bound < 1e-9


def test_reduced_table_he4_matches_oracle_and_golden():
    """He-4: bit-exact against the oracle, and against the stored table whose
    generation checked it exactly mod p against all 1.07e10 terms of the plain sum."""
    _, g, (stats, _) = gpu_table("he4")
    o = O.dedup(oops.nucleus("he4"))
    for k in ("rep", "w", "ids"):
        assert np.array_equal(g[k], o[k])
    assert stats == o["stats"]
    tab, info = make_tables.load("he4")
    assert make_tables.digest(g["rep"], g["w"], g["ids"]) == info["sha256"]
    assert list(stats) == info["stats"]


def test_reduced_table_independent_of_seed_and_sites():
    ref = gpu_table("he3", seed=1)[1]
    for seed, sites in ((2, 1), (12345, 2), (99, 3)):
        g = gpu_table("he3", seed=seed, sites=sites)[1]
        for k in ("rep", "w", "ids"):
            assert np.array_equal(g[k], ref[k])


def test_terms_save_load_roundtrip(tmp_path):
    terms, g, _ = gpu_table("deuteron")
    p = str(tmp_path / "deuteron.wick")
    terms.save(p)
    t2 = wick.Terms.load_file(p)
    g2 = t2.copy()
    for k in ("rep", "w", "ids"):
        assert np.array_equal(g[k], g2[k])
    raw = bytearray(open(p, "rb").read())
    raw[-20] ^= 0x55                                     # corrupt one byte of the arrays
    open(p, "wb").write(bytes(raw))
    with pytest.raises(wick.WickError) as e:
        wick.Terms.load_file(p)
    assert e.value.code == wick.WICK_EIO


# ---------------------------------------------------------------------------
# correlators
# ---------------------------------------------------------------------------
def test_deuteron_workload_fp64():
    """L=4, T=8, one source, complex128: the plain FP64 path against the raw Wick sum."""
    w = synth.WORKLOADS["deuteron"]
    Su, Sd = props(w["L"], w["T"], w["n_src"], seed=w["seed"])
    terms, _, _ = gpu_table("deuteron")
    tabs = wick.Tables(operators.nucleus("deuteron"))
    C = gpu_contract(gpu_blocks(Su, Sd, tabs, "fp64"), terms, "fp64")
    onuc = oops.nucleus("deuteron")
    ref = O.raw_correlator(onuc, O.blocks_single(Su, Sd, onuc))
    assert rel_per_t(C, ref) < FP64_TOL


def test_he3_workload_fp64():
    """L=8, T=16, two sources: every slice against the oracle's reduced sum, two
    slices against the raw Wick sum over all 2e7 terms."""
    w = synth.WORKLOADS["he3"]
    Su, Sd = props(w["L"], w["T"], w["n_src"], seed=w["seed"])
    terms, _, _ = gpu_table("he3")
    tabs = wick.Tables(operators.nucleus("he3"))
    C = gpu_contract(gpu_blocks(Su, Sd, tabs, "fp64"), terms, "fp64")
    onuc = oops.nucleus("he3")
    Bh = O.blocks_single(Su, Sd, onuc)
    ref = O.table_correlator(onuc, Bh, O.dedup(onuc))
    assert rel_per_t(C, ref) < FP64_TOL
    raw = O.raw_correlator(onuc, Bh[:, :1])
    assert rel_per_t(C[:, :1], raw) < FP64_TOL


@pytest.fixture(scope="module")
def he4_case():
    w = synth.WORKLOADS["he4"]
    Su, Sd = props(w["L"], w["T"], w["n_src"], seed=w["seed"], dtype=np.complex64)
    tab = O.dedup(oops.nucleus("he4"))
    terms, _, _ = gpu_table("he4")
    return Su, Sd, tab, terms


HE4_SAMPLES = [(0, 0), (1, 7), (3, 31)]   # (src, t) slices checked against the oracle


@pytest.mark.parametrize("precision,tol", [("mixed", MIXED_TOL), ("fp64", FP64_TOL)])
def test_he4_workload(he4_case, precision, tol):
    """L=16, T=32, four sources, complex64 storage (the benchmark's launch
    configuration); sampled slices against the oracle."""
    Su, Sd, tab, terms = he4_case
    tabs = wick.Tables(operators.nucleus("he4"))
    B = gpu_blocks(Su, Sd, tabs, precision)
    C = gpu_contract(B, terms, precision)
    onuc = oops.nucleus("he4")
    Bn = B.cpu().numpy()
    for s, t in HE4_SAMPLES:
        Bh = O.blocks_single(Su[s:s + 1, t:t + 1].astype(np.complex128), Sd[s:s + 1, t:t + 1].astype(np.complex128),
                             onuc)
        assert block_err(Bn[s:s + 1, t:t + 1], O.antisymmetric_blocks(Bh, onuc)) < tol
        ref = O.table_correlator(onuc, Bh, tab)
        assert rel_per_t(C[s:s + 1, t:t + 1], ref) < tol, (s, t)


def test_top_fraction_selection():
    """Evaluating only the largest-weight terms (Sec. V.C) through wick_terms_select."""
    Su, Sd = props(4, 4, 1, seed=21)
    terms, g, _ = gpu_table("he3")
    o = O.dedup(oops.nucleus("he3"))
    thr = np.sort(np.abs(o["w"]))[-len(o["w"]) // 10]
    keep_o = np.abs(o["w"]) >= thr
    sub = dict(ids=o["ids"][keep_o], w=o["w"][keep_o])
    perm = np.nonzero(np.abs(g["w"]) >= thr)[0][::-1]    # any order: the table re-sorts
    terms.select(perm)
    assert terms.count == int(keep_o.sum())
    tabs = wick.Tables(operators.nucleus("he3"))
    C = gpu_contract(gpu_blocks(Su, Sd, tabs, "fp64"), terms, "fp64")
    onuc = oops.nucleus("he3")
    ref = O.table_correlator(onuc, O.blocks_single(Su, Sd, onuc), sub)
    assert rel_per_t(C, ref) < FP64_TOL


@pytest.mark.parametrize("name,fraction", [("he3", 0.05), ("he4", 0.01)])
def test_top_fraction_by_contribution(name, fraction):
    """Sec. V.C as the paper does it: rank the terms by their contribution on a small lattice (a few
    time slices), keep the top fraction, evaluate those on another configuration.  Magnitudes, the
    kept set and the truncated correlator against the oracle."""
    onuc = oops.nucleus(name)
    tabs = wick.Tables(operators.nucleus(name))
    terms, _, _ = gpu_table(name)
    o = O.dedup(onuc)
    # ranking lattice: L=2, three time slices
    Su, Sd = props(2, 3, 1, seed=0x70F)
    Bh = O.blocks_single(Su, Sd, onuc)
    mag_ref = np.abs(O.term_contributions(onuc, Bh, o)).sum(axis=1)
    mag = terms.magnitudes(gpu_blocks(Su, Sd, tabs, "fp64"), 3)
    assert np.max(np.abs(mag - mag_ref) / np.max(mag_ref)) < FP64_TOL
    keep = O.top_terms(mag_ref, fraction)
    terms.top(mag, fraction)
    got = terms.copy()
    assert terms.count == len(keep)
    assert np.array_equal(got["ids"], o["ids"][keep]) and np.array_equal(got["w"], o["w"][keep])
    # evaluation lattice: another configuration
    Su2, Sd2 = props(4, 2, 1, seed=0x710)
    C = gpu_contract(gpu_blocks(Su2, Sd2, tabs, "fp64"), terms, "fp64")
    ref = O.table_correlator(onuc, O.blocks_single(Su2, Sd2, onuc), dict(ids=o["ids"][keep], w=o["w"][keep]))
    assert rel_per_t(C, ref) < FP64_TOL


def test_contract_deterministic():
    Su, Sd = props(4, 4, 2, seed=4)
    terms, _, _ = gpu_table("he3")
    tabs = wick.Tables(operators.nucleus("he3"))
    B = gpu_blocks(Su, Sd, tabs, "fp64")
    a = gpu_contract(B, terms, "mixed")
    b = gpu_contract(B, terms, "mixed")
    assert np.array_equal(a, b)


def test_invalid_arguments_rejected():
    tabs = wick.Tables(operators.nucleus("deuteron"))
    S = torch.zeros((1, 1, 8, 144), dtype=torch.complex128, device="cuda")
    out = torch.zeros((1, 1, tabs.nuc.n_blk), dtype=torch.complex128, device="cuda")
    with pytest.raises(wick.WickError) as e:
        wick.wick_build_blocks(S, S, tabs, 7, out, 2, 1, 1)          # unknown precision
    assert e.value.code == wick.WICK_EINVAL
    S64 = S.to(torch.complex64)
    with pytest.raises(wick.WickError):
        wick.wick_build_blocks(S, S64, tabs, wick.WICK_FP64, out, 2, 1, 1)  # mixed storage types
