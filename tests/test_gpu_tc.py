"""GPU parity of the tensor-core block build (WICK_MIXED on the upper-spin
tables) against the CPU reference and against the CUDA-core double-FP32 kernel.

The tensor-core stage evaluates the update sum over sites as an exact sliced
product: every 16-site chunk is exact in the tensor core's FP32 accumulator and
the slice pairs it drops lie below 2^-35 of the chunk's row/column scales, so
the blocks agree with the FP64 reference to about 1e-11 of each slice's
largest entry.  The tests hold it to 1e-10 (well inside the mixed contract of
1e-6 per time slice of the correlator) and check the device status word.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import operators as oops  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2411_08962_gb300 import build, operators, synth, wick  # noqa: E402

pytestmark = pytest.mark.gpu

TC_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    wick.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def blocks(Su, Sd, nuc, precision, L):
    n_src, T = Su.shape[:2]
    out = torch.empty((n_src, T, nuc.n_blk), dtype=torch.complex128, device="cuda")
    wick.wick_build_blocks(dev(Su), dev(Sd), wick.Tables(nuc), precision, out, L, T, n_src)
    torch.cuda.synchronize()
    assert wick.wick_status() == 0
    return out.cpu().numpy()


def block_err(gpu, ref):
    ref = ref.reshape(gpu.shape)
    scale = np.max(np.abs(ref), axis=-1, keepdims=True)
    return np.max(np.abs(gpu - ref) / scale)


def as_float(S):
    """The values WICK_MIXED computes with: propagator entries rounded to complex64."""
    return S.astype(np.complex64).astype(np.complex128)


def props(L, T, n_src, seed, dtype):
    return (synth.propagator(seed, 0, L, T, n_src, dtype=dtype), synth.propagator(seed, 1, L, T, n_src, dtype=dtype))


@pytest.fixture(params=[0, 1], ids=["pair_kernel", "one_type_per_cta"])
def pair_mode(request):
    """Both tensor-core kernels of the upper-spin tables: the pair kernel (one CTA builds the proton and
    the neutron types from one computation of the diquark values) and one block type per CTA."""
    wick.wick_set_tuning({"no_pair_kernel": request.param})
    yield request.param
    wick.wick_set_tuning(None)


@pytest.mark.parametrize("L,T,n_src,dtype", [
    (1, 1, 1, np.complex128),   # one site: a chunk with empty sites
    (3, 2, 2, np.complex128),   # 27 sites: full chunks and a ragged one
    (4, 4, 1, np.complex64),    # 64 sites: one TMEM round of full chunks
    (7, 2, 1, np.complex128),   # 343 sites: ragged tail of 7
    (17, 1, 1, np.complex64),   # 4913 sites: several CTAs along sites
])
def test_tc_blocks_match_oracle(L, T, n_src, dtype, pair_mode):
    Su, Sd = props(L, T, n_src, seed=0x7C00 + L, dtype=dtype)
    B = blocks(Su, Sd, operators.nucleus("deuteron"), wick.WICK_MIXED, L)
    onuc = oops.nucleus("deuteron")
    ref = O.antisymmetric_blocks(O.blocks_single(as_float(Su), as_float(Sd), onuc), onuc)
    assert block_err(B, ref) < TC_TOL


def test_pair_and_one_type_kernels_agree():
    """He-4 tables on 8^3 x 3 x 2 sources (four ranges of 128 sites, ragged none): the pair kernel and the
    one-type-per-CTA kernel both within TC_TOL of FP64 and within 1e-10 of each other."""
    L = 8
    Su, Sd = props(L, 3, 2, seed=0x7C33, dtype=np.complex64)
    nuc = operators.nucleus("he4")
    f64 = blocks(Su, Sd, nuc, wick.WICK_FP64, L)
    try:
        wick.wick_set_tuning({"range_sites": 128})
        pair = blocks(Su, Sd, nuc, wick.WICK_MIXED, L)
        wick.wick_set_tuning({"range_sites": 128, "no_pair_kernel": 1})
        one = blocks(Su, Sd, nuc, wick.WICK_MIXED, L)
    finally:
        wick.wick_set_tuning(None)
    assert block_err(pair, f64) < TC_TOL and block_err(one, f64) < TC_TOL
    assert block_err(pair, one) < TC_TOL


def test_tc_matches_cuda_core_kernel():
    """WICK_MIXED (tensor cores) against WICK_MIXED_SIMT and WICK_FP64 on one input."""
    L = 8
    Su, Sd = props(L, 3, 2, seed=0x7C11, dtype=np.complex64)
    nuc = operators.nucleus("he4")
    tc = blocks(Su, Sd, nuc, wick.WICK_MIXED, L)
    simt = blocks(Su, Sd, nuc, wick.WICK_MIXED_SIMT, L)
    f64 = blocks(Su, Sd, nuc, wick.WICK_FP64, L)
    assert block_err(simt, f64) < 1e-11
    assert block_err(tc, f64) < TC_TOL


def test_tc_scale_invariance():
    """The fixed-point grids follow the data: scaling S by 2^k scales B by 2^(3k) exactly."""
    L = 4
    Su, Sd = props(L, 2, 1, seed=0x7C22, dtype=np.complex128)
    nuc = operators.nucleus("deuteron")
    B0 = blocks(Su, Sd, nuc, wick.WICK_MIXED, L)
    for k in (-20, 9):
        Bk = blocks(Su * 2.0 ** k, Sd * 2.0 ** k, nuc, wick.WICK_MIXED, L)
        assert np.array_equal(Bk, B0 * 2.0 ** (3 * k))


def test_tc_zero_and_sparse_input():
    """All-zero propagators give zero blocks; a single non-zero site gives that site's blocks."""
    L = 3
    z = np.zeros((1, 1, L ** 3, 3, 4, 3, 4), dtype=np.complex128)
    nuc = operators.nucleus("deuteron")
    assert not np.any(blocks(z, z, nuc, wick.WICK_MIXED, L))
    Su, Sd = props(L, 1, 1, seed=0x7C33, dtype=np.complex128)
    Su[:, :, 1:] = 0
    B = blocks(Su, Sd, nuc, wick.WICK_MIXED, L)
    onuc = oops.nucleus("deuteron")
    ref = O.antisymmetric_blocks(O.blocks_single(as_float(Su), as_float(Sd), onuc), onuc)
    assert block_err(B, ref) < TC_TOL


def test_tc_deterministic():
    L = 8
    Su, Sd = props(L, 2, 1, seed=0x7C44, dtype=np.complex64)
    nuc = operators.nucleus("deuteron")
    assert np.array_equal(blocks(Su, Sd, nuc, wick.WICK_MIXED, L), blocks(Su, Sd, nuc, wick.WICK_MIXED, L))


def test_mixed_simt_rejected_by_contract():
    """WICK_MIXED_SIMT selects a block kernel; the contraction takes FP64 or MIXED only."""
    nuc = operators.nucleus("deuteron")
    terms = wick.wick_reduce_terms(wick.Tables(nuc), 0x2411, 2, 1)
    Bk = torch.zeros((1, 1, nuc.n_blk), dtype=torch.complex128, device="cuda")
    C = torch.empty((1, 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(wick.WickError):
        wick.wick_contract(Bk, 1, 1, terms, wick.WICK_MIXED_SIMT, C)


@pytest.mark.parametrize("L,T,dtype", [
    (2, 2, np.complex64),       # 8 sites: one chunk
    (3, 1, np.complex128),      # 27 sites: ragged chunk, complex128 staging
    (9, 1, np.complex64),       # 729 sites: two site ranges, six rounds of 128
])
def test_tc_full_spin_blocks_match_oracle(L, T, dtype):
    """Full-spin p+-/n+- blocks (four M tiles, five column tiles) against the CPU reference."""
    nuc = operators.cluster("triton")
    Su, Sd = props(L, T, 1, seed=0x7C55 + L, dtype=dtype)
    B = blocks(Su, Sd, nuc, wick.WICK_MIXED, L)
    onuc = oops.triton_cluster()
    ref = O.antisymmetric_blocks(O.blocks_single(as_float(Su), as_float(Sd), onuc), onuc)
    assert block_err(B, ref) < TC_TOL


def test_tc_full_spin_matches_cuda_core_kernel():
    L = 6
    Su, Sd = props(L, 2, 1, seed=0x7C66, dtype=np.complex64)
    nuc = operators.cluster("he4_cluster")
    tc = blocks(Su, Sd, nuc, wick.WICK_MIXED, L)
    f64 = blocks(Su, Sd, nuc, wick.WICK_FP64, L)
    assert block_err(blocks(Su, Sd, nuc, wick.WICK_MIXED_SIMT, L), f64) < 1e-11
    assert block_err(tc, f64) < TC_TOL
