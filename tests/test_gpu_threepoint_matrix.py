"""GPU parity of the plane-wave three-point function, the correlation matrix and the plane-wave
2H operator of Eq. NP_op, through the C ABI against the CPU reference.

* derivative blocks (wick_build_blocks_3pt) against the oracle's: the linear coefficient of the
  single-product blocks in the direction Sig, antisymmetrised (blocks are at most quadratic in
  one flavour, so three evaluations at the cube roots of unity give it exactly);
* three-point functions (wick_contract_3pt): deuteron and He-4, current on u and on d, FP64
  <= 1e-12 and mixed <= 1e-6 per time slice against the oracle's coefficient extraction;
* the 3 x 3 correlation matrix of three plane-wave deuteron operators (wick_reduce_terms_matrix,
  Eqs. E1-E3): every element against the oracle's (sink i, source j) correlator; the merged table
  is smaller than the elements' tables together;
* Eq. NP_op with a plane-wave sink (full-spin blocks, the tensor-core build for mixed): the
  reduced table bit-exact and the correlator within the tolerances.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import operators as oops  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2411_08962_gb300 import build, operators, synth, wick  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-6
PREC = {"fp64": (wick.WICK_FP64, FP64_TOL), "mixed": (wick.WICK_MIXED, MIXED_TOL)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    wick.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def props(L, T, n_src, seed, precision="fp64"):
    """(Su, Sd, Sig); for the mixed path complex64 values (what that path computes with), held as
    complex128 so that the oracle sees the same numbers."""
    out = tuple(synth.propagator(seed, f, L, T, n_src) for f in (0, 1)) + (synth.propagator(seed + 7, 0, L, T, n_src),)
    if precision == "mixed":
        out = tuple(a.astype(np.complex64).astype(np.complex128) for a in out)
    return out


def rel_per_t(a, b):
    return np.max(np.abs(a - b) / np.abs(b))


def oracle_dblocks(Su, Sd, Sig, flavour, onuc):
    acc = 0.0
    for k in range(3):
        e = np.exp(2j * np.pi * k / 3)
        su = Su + e * Sig if flavour == 0 else Su
        sd = Sd + e * Sig if flavour == 1 else Sd
        acc = acc + O.antisymmetric_blocks(O.blocks_single(su, sd, onuc), onuc) * np.conj(e)
    return acc / 3


def gpu_3pt(Su, Sd, Sig, flavour, tabs, terms, prec):
    n_src, T, V = Su.shape[:3]
    L = round(V ** (1 / 3))
    nb = tabs.nuc.n_blk
    B = torch.empty((n_src, T, nb), dtype=torch.complex128, device="cuda")
    D = torch.empty_like(B)
    wick.wick_build_blocks(dev(Su), dev(Sd), tabs, prec, B, L, T, n_src)
    wick.wick_build_blocks_3pt(dev(Su), dev(Sd), dev(Sig), flavour, tabs, prec, D, L, T, n_src)
    C = torch.empty((n_src, T), dtype=torch.complex128, device="cuda")
    wick.wick_contract_3pt(B, D, n_src, T, terms, prec, C)
    torch.cuda.synchronize()
    return D.cpu().numpy(), C.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("flavour", [wick.WICK_U, wick.WICK_D])
def test_three_point_deuteron(precision, flavour):
    prec, tol = PREC[precision]
    Su, Sd, Sig = props(3, 2, 2, seed=0x3A01, precision=precision)
    tabs = wick.Tables(operators.nucleus("deuteron"))
    terms = wick.wick_reduce_terms(tabs)
    D, C = gpu_3pt(Su, Sd, Sig, flavour, tabs, terms, prec)
    onuc = oops.nucleus("deuteron")
    Dref = oracle_dblocks(Su, Sd, Sig, flavour, onuc)
    scale = np.max(np.abs(Dref), axis=-1, keepdims=True)
    assert np.max(np.abs(D - Dref) / scale) < (1e-13 if precision == "fp64" else 1e-9)
    ref = O.three_point_planewave(Su, Sd, Sig, flavour, onuc)
    assert rel_per_t(C, ref) < tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_three_point_he4(precision):
    prec, tol = PREC[precision]
    Su, Sd, Sig = props(2, 2, 1, seed=0x3A04, precision=precision)
    tabs = wick.Tables(operators.nucleus("he4"))
    terms = wick.wick_reduce_terms(tabs)
    onuc = oops.nucleus("he4")
    tab = O.dedup(onuc)
    for flavour in (wick.WICK_U, wick.WICK_D):
        _, C = gpu_3pt(Su, Sd, Sig, flavour, tabs, terms, prec)
        ref = O.three_point_planewave(Su, Sd, Sig, flavour, onuc, tab)
        assert rel_per_t(C, ref) < tol, flavour


def test_three_point_euler_on_the_gpu():
    """Sig = S_u: the three-point function is n_u times the correlator (Euler's identity)."""
    Su, Sd, _ = props(3, 2, 1, seed=0x3A05)
    tabs = wick.Tables(operators.nucleus("he3"))
    terms = wick.wick_reduce_terms(tabs)
    _, C3 = gpu_3pt(Su, Sd, Su, wick.WICK_U, tabs, terms, wick.WICK_FP64)
    B = torch.empty((1, 2, tabs.nuc.n_blk), dtype=torch.complex128, device="cuda")
    wick.wick_build_blocks(dev(Su), dev(Sd), tabs, wick.WICK_FP64, B, 3, 2, 1)
    C = torch.empty((1, 2), dtype=torch.complex128, device="cuda")
    wick.wick_contract(B, 1, 2, terms, wick.WICK_FP64, C)
    torch.cuda.synchronize()
    assert rel_per_t(C3, 5 * C.cpu().numpy()) < FP64_TOL      # He-3: five u quarks


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_correlation_matrix(precision):
    prec, tol = PREC[precision]
    L, T, n_src = 3, 3, 2
    Su, Sd, _ = props(L, T, n_src, seed=0x3A06, precision=precision)
    basis = operators.deuteron_pw_basis()
    tl = [wick.Tables(n) for n in basis]
    mt = wick.wick_reduce_terms_matrix(tl)
    assert mt.elements == 9
    sizes = [wick.wick_reduce_terms(wick.Tables(
        operators.Nucleus("el", 2, basis[i].ops, 2, basis[i].chi, basis[i].sink, basis[j].src, basis[i].src_flav)
    )).count for i in range(3) for j in range(3)]
    assert max(sizes) <= mt.count < sum(sizes)            # shared products are one term
    B = torch.empty((n_src, T, tl[0].nuc.n_blk), dtype=torch.complex128, device="cuda")
    wick.wick_build_blocks(dev(Su), dev(Sd), tl[0], prec, B, L, T, n_src)
    C = torch.empty((9, n_src, T), dtype=torch.complex128, device="cuda")
    wick.wick_contract(B, n_src, T, mt, prec, C)
    torch.cuda.synchronize()
    Cn = C.cpu().numpy()
    ob = oops.deuteron_pw_basis()
    for i in range(3):
        for j in range(3):
            ref = O.correlator(Su, Sd, O.matrix_element(ob[i], ob[j]))
            assert rel_per_t(Cn[i * 3 + j], ref) < tol, (i, j)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_np_operator_planewave(precision):
    prec, tol = PREC[precision]
    L, T, n_src = 3, 2, 1
    Su, Sd, _ = props(L, T, n_src, seed=0x3A07)
    tabs = wick.Tables(operators.deuteron_np())
    terms = wick.wick_reduce_terms(tabs, seed=0x77)
    onuc = oops.deuteron_np_planewave()
    o = O.dedup(onuc)
    g = terms.copy()
    for k in ("rep", "w", "ids"):
        assert np.array_equal(g[k], o[k]), k
    B = torch.empty((n_src, T, tabs.nuc.n_blk), dtype=torch.complex128, device="cuda")
    wick.wick_build_blocks(dev(Su.astype(np.complex64)), dev(Sd.astype(np.complex64)), tabs, prec, B, L, T, n_src)
    C = torch.empty((n_src, T), dtype=torch.complex128, device="cuda")
    wick.wick_contract(B, n_src, T, terms, prec, C)
    torch.cuda.synchronize()
    su, sd = Su.astype(np.complex64).astype(np.complex128), Sd.astype(np.complex64).astype(np.complex128)
    ref = O.correlator(su, sd, onuc)
    assert rel_per_t(C.cpu().numpy(), ref) < tol
