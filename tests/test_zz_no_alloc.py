"""wick_contract_noalloc: the contraction for callers that cannot allocate.

Some callers cannot call cudaMalloc once they are running -- for example an
application whose caching allocator already holds the device memory it may
use, or a runtime that forbids driver-level allocations (and the device-wide
synchronisation they imply) after its set-up phase.  wick_contract allocates
its scratch on first use; wick_contract_noalloc keeps that scratch in a fixed
1 MiB array inside the library instead.  These tests call it through the C ABI
twice in a row, on two different inputs, and check each result against
wick_contract within the tolerance of the parity tests; they check that a
call leaves the device's free memory unchanged, that 65,536 slices (the
array's capacity) are accepted and that one more is refused with
WICK_ESCRATCH.  The file is collected last and passes alone in a fresh
process as well as after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2411_08962_gb300 import build, operators, synth, wick  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12       # FP64 contraction; the double-FP32 one differs from it only by the chunking of the FP64 sums
CAPACITY = 65536  # slices one call may take


def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    wick.load()


@pytest.mark.parametrize("precision", [wick.WICK_FP64, wick.WICK_MIXED], ids=["fp64", "mixed"])
def test_noalloc_contract_matches_contract_on_two_calls(precision):
    _setup()
    L, T, n_src = 4, 4, 2
    tabs = wick.Tables(operators.nucleus("he3"))
    terms = wick.wick_reduce_terms(tabs)
    inputs = []
    for seed in (1234, 5678):
        Su = torch.from_numpy(synth.propagator(seed, 0, L, T, n_src)).cuda()
        Sd = torch.from_numpy(synth.propagator(seed, 1, L, T, n_src)).cuda()
        blocks = torch.empty((n_src, T, tabs.nuc.n_blk), dtype=torch.complex128, device="cuda")
        wick.wick_build_blocks(Su, Sd, tabs, wick.WICK_FP64, blocks, L, T, n_src)
        inputs.append(blocks)
    outs = [torch.full((n_src, T), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
            for _ in inputs]
    torch.cuda.synchronize()
    # the first call may make the driver load the library's device code; the second allocates nothing
    wick.wick_contract_noalloc(inputs[0], n_src, T, terms, precision, outs[0])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    wick.wick_contract_noalloc(inputs[1], n_src, T, terms, precision, outs[1])
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes during a no-alloc call"
    for call, (blocks, got) in enumerate(zip(inputs, outs)):
        ref = torch.empty((n_src, T), dtype=torch.complex128, device="cuda")
        wick.wick_contract(blocks, n_src, T, terms, precision, ref)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g)), f"call {call}: output not written"
        assert np.max(np.abs(g - r) / np.abs(r)) < TOL, f"call {call}"


def test_noalloc_capacity_limit():
    _setup()
    tabs = wick.Tables(operators.nucleus("deuteron"))
    terms = wick.wick_reduce_terms(tabs)
    nb = tabs.nuc.n_blk
    # blocks and outputs sized for every slice of the call, so that nothing could read out of bounds
    g = torch.Generator(device="cuda").manual_seed(7)
    blocks = torch.randn((CAPACITY + 1, nb), dtype=torch.complex128, device="cuda", generator=g)
    ref = torch.empty(CAPACITY + 1, dtype=torch.complex128, device="cuda")
    got = torch.full((CAPACITY + 1,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    wick.wick_contract(blocks, 1, CAPACITY, terms, wick.WICK_FP64, ref)
    wick.wick_contract_noalloc(blocks, 1, CAPACITY, terms, wick.WICK_FP64, got)
    torch.cuda.synchronize()
    r, gg = ref[:CAPACITY].cpu().numpy(), got[:CAPACITY].cpu().numpy()
    assert np.all(np.isfinite(gg))
    assert np.max(np.abs(gg - r) / np.abs(r)) < TOL
    with pytest.raises(wick.WickError) as e:
        wick.wick_contract_noalloc(blocks, 1, CAPACITY + 1, terms, wick.WICK_FP64, got)
    assert e.value.code == wick.WICK_ESCRATCH
    torch.cuda.synchronize()
    assert np.isnan(got[CAPACITY].cpu().numpy()), "the refused call wrote its output"
