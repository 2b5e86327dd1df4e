"""wick_contract_noalloc: the contraction for callers that cannot allocate.

Some callers cannot call cudaMalloc once they are running -- for example an
application whose caching allocator already holds the device memory it may
use, or a runtime that forbids driver-level allocations (and the device-wide
synchronisation they imply) after its set-up phase.  wick_contract allocates
its scratch on first use; wick_contract_noalloc keeps that scratch in a fixed
1 MiB array inside the library instead.  This test calls it through the C ABI
twice in a row, on two different inputs, and checks each result against
wick_contract within the FP64 tolerance of the parity tests.  It lives in a
file of its own, collected last, and passes alone in a fresh process as well
as after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2411_08962_gb300 import build, operators, synth, wick  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def test_noalloc_contract_matches_contract_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    wick.load()
    L, T, n_src = 4, 4, 2
    tabs = wick.Tables(operators.nucleus("he3"))
    terms = wick.wick_reduce_terms(tabs)
    for call, seed in enumerate((1234, 5678)):
        Su = torch.from_numpy(synth.propagator(seed, 0, L, T, n_src)).cuda()
        Sd = torch.from_numpy(synth.propagator(seed, 1, L, T, n_src)).cuda()
        blocks = torch.empty((n_src, T, tabs.nuc.n_blk), dtype=torch.complex128, device="cuda")
        wick.wick_build_blocks(Su, Sd, tabs, wick.WICK_FP64, blocks, L, T, n_src)
        ref = torch.empty((n_src, T), dtype=torch.complex128, device="cuda")
        wick.wick_contract(blocks, n_src, T, terms, wick.WICK_FP64, ref)
        got = torch.full((n_src, T), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        wick.wick_contract_noalloc(blocks, n_src, T, terms, wick.WICK_FP64, got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g)), f"call {call}: output not written"
        assert np.max(np.abs(g - r) / np.abs(r)) < FP64_TOL, f"call {call}"
