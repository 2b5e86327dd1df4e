"""GPU parity for the Li-7 reading: He-4 cluster x triton cluster.

Block types p+, p-, n+, n- (C gamma5 P_pm, all four spins, 27,648 entries per
slice); the He-4 cluster (chibar eta - chi etabar)/sqrt2 and the triton
n_-^T C g5 p_+ n_+^J reduced on the device bit-exactly against the oracle
(the triton table has 1,071,360 terms); Li-7 = product of the two cluster
correlators.  Workload: L=24, T=48, one source, complex64.
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
ORACLE = {"he4_cluster": oops.he4_cluster, "triton": oops.triton_cluster}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    wick.load()


@pytest.fixture(scope="module")
def clusters():
    out = {}
    for name in ORACLE:
        tabs = wick.Tables(operators.cluster(name))
        out[name] = (tabs, wick.wick_reduce_terms(tabs))
    return out


def gpu_blocks(Su, Sd, tabs, prec):
    n_src, T, V = Su.shape[:3]
    L = round(V ** (1 / 3))
    B = torch.empty((n_src, T, tabs.nuc.n_blk), dtype=torch.complex128, device="cuda")
    wick.wick_build_blocks(torch.from_numpy(Su).cuda(), torch.from_numpy(Sd).cuda(), tabs, prec, B, L, T, n_src)
    torch.cuda.synchronize()
    return B


@pytest.mark.parametrize("prec,tol", [(wick.WICK_FP64, FP64_TOL), (wick.WICK_MIXED, MIXED_TOL)])
def test_pm_blocks_match_oracle(clusters, prec, tol):
    tabs = clusters["triton"][0]
    Su = synth.propagator(71, 0, 2, 2, 1, dtype=np.complex64)
    Sd = synth.propagator(71, 1, 2, 2, 1, dtype=np.complex64)
    B = gpu_blocks(Su, Sd, tabs, prec).cpu().numpy()
    onuc = oops.triton_cluster()
    ref = O.antisymmetric_blocks(O.blocks_single(Su.astype(np.complex128), Sd.astype(np.complex128), onuc), onuc)
    scale = np.max(np.abs(ref), axis=-1, keepdims=True)
    assert np.max(np.abs(B - ref) / scale) < tol


@pytest.mark.parametrize("name", list(ORACLE))
def test_cluster_tables_bit_exact(clusters, name):
    g = clusters[name][1].copy()
    stats, bound = clusters[name][1].stats()
    o = O.dedup(ORACLE[name]())
    for k in ("rep", "w", "ids"):
        assert np.array_equal(g[k], o[k]), k
    assert stats == o["stats"] and bound < 1e-6


def test_li7_workload_sampled(clusters):
    w = synth.WORKLOADS["li7"]
    L, T, n_src = w["L"], w["T"], w["n_src"]
    Su = synth.propagator(w["seed"], 0, L, T, n_src, dtype=np.complex64)
    Sd = synth.propagator(w["seed"], 1, L, T, n_src, dtype=np.complex64)
    tabs = clusters["triton"][0]                       # the p+-, n+- blocks serve both clusters
    B = gpu_blocks(Su, Sd, tabs, wick.WICK_MIXED)
    C = {}
    for name in ORACLE:
        C[name] = torch.empty((n_src, T), dtype=torch.complex128, device="cuda")
        wick.wick_contract(B, n_src, T, clusters[name][1], wick.WICK_MIXED, C[name])
    li7 = torch.empty_like(C["triton"])
    wick.wick_cluster_product(C["he4_cluster"], C["triton"], li7)
    torch.cuda.synchronize()
    got = li7.cpu().numpy()
    sl = [(0, 3), (0, 29)]
    su = np.stack([Su[s, t] for s, t in sl])[None].astype(np.complex128)
    sd = np.stack([Sd[s, t] for s, t in sl])[None].astype(np.complex128)
    ref = np.ones(len(sl), dtype=complex)
    for name, make in ORACLE.items():
        onuc = make()
        ref = ref * O.table_correlator(onuc, O.blocks_single(su, sd, onuc), O.dedup(onuc))[0]
    for q, (s, t) in enumerate(sl):
        assert abs(got[s, t] - ref[q]) / abs(ref[q]) < MIXED_TOL, (s, t)
