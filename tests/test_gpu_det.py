"""GPU parity of the point-sink determinant path (Eq. 2.9, Eq. a1) against the CPU reference.

* The minimal sets zeta_u, zeta_d and Theta the library finds by identity
  testing mod 2^61 - 1 are exactly the reference's (bit-exact integers).
* The FP64 correlator agrees with the reference within 1e-12 relative per time
  slice (2H, 3He on small lattices including ragged site chunks; 4He on one
  site), for complex128 and complex64 storage.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import det as DT  # noqa: E402
from paper_2411_08962_gb300 import build, operators, synth, wick  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    wick.load()


_PLANS = {}


def plan(name):
    if name not in _PLANS:
        _PLANS[name] = wick.DetPlan(operators.point_operator(name))
    return _PLANS[name]


def gpu_point(name, Su, Sd):
    n_src, T, V = Su.shape[:3]
    L = round(V ** (1 / 3))
    out = torch.empty((n_src, T), dtype=torch.complex128, device="cuda")
    wick.wick_det_contract(torch.from_numpy(np.ascontiguousarray(Su)).cuda(),
                           torch.from_numpy(np.ascontiguousarray(Sd)).cuda(), plan(name), out, L, T, n_src)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def props(L, T, n_src, seed, dtype=np.complex128):
    return (synth.propagator(seed, 0, L, T, n_src, dtype=dtype), synth.propagator(seed, 1, L, T, n_src, dtype=dtype))


@pytest.mark.parametrize("name", ["deuteron", "he3"])
def test_minimal_sets_bit_exact(name):
    tab, nu, nd, _ = DT.operator(name)
    zu, zd, th = DT.minimal_sets(tab, tab, nu)
    p = plan(name)
    st = p.stats()
    assert (st["n_u"], st["n_d"]) == (nu, nd)
    assert (st["zeta_u"], st["zeta_d"], st["theta"]) == (len(zu), len(zd), len(th))
    c = p.copy()
    gu = [(tuple(r), tuple(q)) for r, q in zip(c["zu_rows"].tolist(), c["zu_cols"].tolist())]
    gd = [(tuple(r), tuple(q)) for r, q in zip(c["zd_rows"].tolist(), c["zd_cols"].tolist())]
    got = {(gu[k], gd[l]): w for k, l, w in zip(c["k"].tolist(), c["l"].tolist(), c["w"].tolist())}
    ref = {(zu[k], zd[l]): w for (k, l), w in th.items()}
    assert got == ref


@pytest.mark.parametrize("name,L,T,n_src,dtype", [
    ("deuteron", 2, 2, 1, np.complex128),
    ("deuteron", 3, 1, 2, np.complex64),    # 27 sites: one ragged chunk
    ("deuteron", 4, 1, 1, np.complex128),   # 64 sites: two chunks
    ("he3", 2, 1, 1, np.complex128),
    ("he4", 1, 1, 1, np.complex128),
])
def test_point_correlator_matches_oracle(name, L, T, n_src, dtype):
    Su, Sd = props(L, T, n_src, seed=0xD37 + L, dtype=dtype)
    tab, nu, nd, scale = DT.operator(name)
    ref = DT.point_correlator(Su.astype(np.complex128), Sd.astype(np.complex128), tab, tab, nu, nd, scale)
    got = gpu_point(name, Su, Sd)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < FP64_TOL


def test_point_correlator_deterministic():
    Su, Sd = props(3, 2, 1, seed=0xD38)
    assert np.array_equal(gpu_point("deuteron", Su, Sd), gpu_point("deuteron", Su, Sd))


def test_invalid_operator_rejected():
    q = operators.point_operator("deuteron")
    bad = operators.QuarkOperator("bad", q.n_u, q.n_d, q.chi.copy(), q.w.copy())
    bad.chi[0, 0] = 12
    with pytest.raises(wick.WickError):
        wick.DetPlan(bad)
    with pytest.raises(wick.WickError):
        wick.DetPlan(q, operators.point_operator("he3"))   # different quark content


def basis_plan():
    if "basis" not in _PLANS:
        _PLANS["basis"] = wick.DetPlan(None, matrix=operators.deuteron_basis())
    return _PLANS["basis"]


def gpu_matrix(Su, Sd):
    n_src, T, V = Su.shape[:3]
    L = round(V ** (1 / 3))
    p = basis_plan()
    n_el = p.stats()["n_el"]
    out = torch.empty((n_el, n_src, T), dtype=torch.complex128, device="cuda")
    wick.wick_det_contract(torch.from_numpy(np.ascontiguousarray(Su)).cuda(),
                           torch.from_numpy(np.ascontiguousarray(Sd)).cuda(), p, out, L, T, n_src)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_correlation_matrix_matches_oracle():
    """C_ij = <O_i(t) Obar_j(0)> for the three 2H operators (Eq. E3), every element."""
    from oracle import operators as oops
    basis = oops.deuteron_basis()
    Su, Sd = props(2, 2, 1, seed=0xD39)
    got = gpu_matrix(Su, Sd)
    assert got.shape[0] == 9
    for i, (ti, _) in enumerate(basis):
        for j, (tj, _) in enumerate(basis):
            ref = DT.point_correlator(Su, Sd, ti, tj, 3, 3)
            assert np.max(np.abs(got[3 * i + j] - ref) / np.abs(ref)) < FP64_TOL


def test_correlation_matrix_shares_determinants():
    """One minimal set for all nine elements; each element's Theta is the pair's, bit-exact."""
    from oracle import operators as oops
    basis = oops.deuteron_basis()
    p = basis_plan()
    c, off = p.copy(), p.element_offsets()
    gu = [(tuple(r), tuple(q)) for r, q in zip(c["zu_rows"].tolist(), c["zu_cols"].tolist())]
    gd = [(tuple(r), tuple(q)) for r, q in zip(c["zd_rows"].tolist(), c["zd_cols"].tolist())]
    union_u, union_d = set(), set()
    for i, (ti, _) in enumerate(basis):
        for j, (tj, _) in enumerate(basis):
            zu, zd, th = DT.minimal_sets(ti, tj, 3)
            union_u |= {zu[k] for k, _ in th}
            union_d |= {zd[l] for _, l in th}
            e0, e1 = off[3 * i + j], off[3 * i + j + 1]
            got = {(gu[k], gd[l]): w for k, l, w in zip(c["k"][e0:e1].tolist(), c["l"][e0:e1].tolist(),
                                                         c["w"][e0:e1].tolist())}
            assert got == {(zu[k], zd[l]): w for (k, l), w in th.items()}
    assert set(gu) == union_u and set(gd) == union_d


def test_matrix_diagonal_equals_single_correlator():
    Su, Sd = props(3, 1, 1, seed=0xD3A)
    got = gpu_matrix(Su, Sd)
    single = gpu_point("deuteron", Su, Sd)   # n^T (C g5 P+) p
    assert np.max(np.abs(got[0] - single) / np.abs(single)) < 1e-13


@pytest.mark.parametrize("name,flavour,L", [("deuteron", wick.WICK_U, 2), ("deuteron", wick.WICK_D, 3),
                                           ("he3", wick.WICK_D, 1)])
def test_three_point_matches_oracle(name, flavour, L):
    """Current on u or d through a sequential propagator: the derivative of Eq. 2.9 (FP64, 1e-12)."""
    T, n_src = 2, 1
    Su, Sd = props(L, T, n_src, seed=0xD3B + L)
    Sig = synth.propagator(0xD3C, 0, L, T, n_src)
    tab, nu, nd, scale = DT.operator(name)
    ref = DT.point_3pt(Su, Sd, Sig, flavour, tab, tab, nu, nd, scale)
    out = torch.empty((n_src, T), dtype=torch.complex128, device="cuda")
    dev_ = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (Su, Sd, Sig)]
    wick.wick_det_contract_3pt(dev_[0], dev_[1], dev_[2], flavour, plan(name), out, L, T, n_src)
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy() - ref) / np.abs(ref)) < FP64_TOL


def test_three_point_euler_identity_on_gpu():
    """Sigma_u = S_u gives n_u times the two-point function."""
    Su, Sd = props(3, 1, 1, seed=0xD3D)
    out = torch.empty((1, 1), dtype=torch.complex128, device="cuda")
    su, sd = torch.from_numpy(Su).cuda(), torch.from_numpy(Sd).cuda()
    wick.wick_det_contract_3pt(su, sd, su, wick.WICK_U, plan("deuteron"), out, 3, 1, 1)
    two = gpu_point("deuteron", Su, Sd)
    assert np.max(np.abs(out.cpu().numpy() - 3 * two) / np.abs(two)) < 1e-13


# ---------------------------------------------------------------------------
# WICK_MIXED: minor tables, determinants and the Theta sum in double-FP32 on the float pipes
# ---------------------------------------------------------------------------
MIXED_TOL = 1e-9


def gpu_point_mixed(name, Su, Sd):
    n_src, T, V = Su.shape[:3]
    L = round(V ** (1 / 3))
    out = torch.empty((n_src, T), dtype=torch.complex128, device="cuda")
    wick.wick_det_contract(torch.from_numpy(np.ascontiguousarray(Su)).cuda(),
                           torch.from_numpy(np.ascontiguousarray(Sd)).cuda(), plan(name), out, L, T, n_src,
                           precision=wick.WICK_MIXED)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("name,L,T,n_src,dtype", [
    ("deuteron", 3, 1, 2, np.complex64),    # 27 sites: ragged chunks
    ("deuteron", 2, 2, 1, np.complex128),   # complex128 input split into float pairs
    ("he3", 2, 1, 1, np.complex64),         # 5 x 5 through the 3 x 3 minor table
    ("he4", 1, 1, 1, np.complex64),         # 6 x 6 through the 3 x 3 minor table
])
def test_point_correlator_mixed_matches_oracle(name, L, T, n_src, dtype):
    Su, Sd = props(L, T, n_src, seed=0xD40 + L, dtype=dtype)
    tab, nu, nd, scale = DT.operator(name)
    ref = DT.point_correlator(Su.astype(np.complex128), Sd.astype(np.complex128), tab, tab, nu, nd, scale)
    got = gpu_point_mixed(name, Su, Sd)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < MIXED_TOL


def test_matrix_mixed_matches_fp64():
    Su, Sd = props(2, 1, 1, seed=0xD41, dtype=np.complex64)
    p = basis_plan()
    n_el = p.stats()["n_el"]
    su, sd = torch.from_numpy(Su).cuda(), torch.from_numpy(Sd).cuda()
    outs = []
    for prec in (wick.WICK_FP64, wick.WICK_MIXED):
        out = torch.empty((n_el, 1, 1), dtype=torch.complex128, device="cuda")
        wick.wick_det_contract(su, sd, p, out, 2, 1, 1, precision=prec)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    assert np.max(np.abs(outs[1] - outs[0]) / np.abs(outs[0])) < MIXED_TOL


@pytest.mark.parametrize("flavour", [wick.WICK_U, wick.WICK_D])
def test_three_point_mixed_matches_oracle(flavour):
    L, T, n_src = 2, 1, 1
    Su, Sd = props(L, T, n_src, seed=0xD42, dtype=np.complex64)
    Sig = synth.propagator(0xD43, 0, L, T, n_src, dtype=np.complex64)
    tab, nu, nd, scale = DT.operator("deuteron")
    ref = DT.point_3pt(Su.astype(np.complex128), Sd.astype(np.complex128), Sig.astype(np.complex128), flavour,
                       tab, tab, nu, nd, scale)
    out = torch.empty((n_src, T), dtype=torch.complex128, device="cuda")
    dev_ = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (Su, Sd, Sig)]
    wick.wick_det_contract_3pt(dev_[0], dev_[1], dev_[2], flavour, plan("deuteron"), out, L, T, n_src,
                               precision=wick.WICK_MIXED)
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy() - ref) / np.abs(ref)) < MIXED_TOL


def test_three_point_mixed_rejects_large_flavour():
    """The double-FP32 derivative exists in the cofactor form (n_f <= 3) only: 3He's d quarks (4) refuse."""
    Su, Sd = props(1, 1, 1, seed=0xD44, dtype=np.complex64)
    out = torch.empty((1, 1), dtype=torch.complex128, device="cuda")
    su, sd = torch.from_numpy(Su).cuda(), torch.from_numpy(Sd).cuda()
    with pytest.raises(wick.WickError):
        wick.wick_det_contract_3pt(su, sd, su, wick.WICK_D, plan("he3"), out, 1, 1, 1, precision=wick.WICK_MIXED)


def test_deuteron_benchmark_size_matches_oracle():
    """2H on the 24^3 lattice of the point-sink benchmark (one time slice, complex64 storage, the
    benchmark's launch configuration): FP64 within 1e-12 and double-FP32 within 1e-9 of the oracle."""
    L, T, n_src = 24, 1, 1
    Su, Sd = props(L, T, n_src, seed=0xD45, dtype=np.complex64)
    tab, nu, nd, scale = DT.operator("deuteron")
    ref = DT.point_correlator(Su.astype(np.complex128), Sd.astype(np.complex128), tab, tab, nu, nd, scale)
    assert np.max(np.abs(gpu_point("deuteron", Su, Sd) - ref) / np.abs(ref)) < FP64_TOL
    assert np.max(np.abs(gpu_point_mixed("deuteron", Su, Sd) - ref) / np.abs(ref)) < MIXED_TOL


def test_he3_benchmark_size_matches_oracle():
    """3He on the 8^3 lattice of the point-sink benchmark (one time slice): 5 x 5 determinants through
    the 3 x 3 minor table, FP64 within 1e-12 and double-FP32 within 1e-9 of the oracle."""
    L, T, n_src = 8, 1, 1
    Su, Sd = props(L, T, n_src, seed=0xD46, dtype=np.complex64)
    tab, nu, nd, scale = DT.operator("he3")
    ref = DT.point_correlator(Su.astype(np.complex128), Sd.astype(np.complex128), tab, tab, nu, nd, scale)
    assert np.max(np.abs(gpu_point("he3", Su, Sd) - ref) / np.abs(ref)) < FP64_TOL
    assert np.max(np.abs(gpu_point_mixed("he3", Su, Sd) - ref) / np.abs(ref)) < MIXED_TOL
