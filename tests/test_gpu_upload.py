"""Upload of the propagator rows a block build reads (wick_upload_rows), by the
copy engines and by the gather kernel.

The block build (Eq. 2.4/2.5) reads S(x)(chi, c) only at the sink indices of
the nucleon tables.  Rows uploaded alone into a device buffer whose other rows
hold NaN must give the same blocks, bit for bit, as the fully copied
propagator (tensor-core mixed, CUDA-core mixed and FP64 paths), and the byte
count must be exactly those rows.
"""
import ctypes

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


def blocks(Su, Sd, tabs, nuc, precision, L, T, n_src):
    out = torch.empty((n_src, T, nuc.n_blk), dtype=torch.complex128, device="cuda")
    wick.wick_build_blocks(Su, Sd, tabs, precision, out, L, T, n_src)
    torch.cuda.synchronize()
    assert wick.wick_status() == 0
    return out.cpu().numpy()


@pytest.mark.parametrize("mode", [wick.WICK_UPLOAD_DMA, wick.WICK_UPLOAD_KERNEL, wick.WICK_UPLOAD_AUTO])
@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("name", ["he4", "deuteron"])
def test_uploaded_rows_give_identical_blocks(name, dtype, mode):
    L, T, n_src = 4, 3, 2
    nuc = operators.nucleus(name)
    tabs = wick.Tables(nuc)
    hu = torch.from_numpy(synth.propagator(0x51, 0, L, T, n_src, dtype=dtype)).pin_memory()
    hd = torch.from_numpy(synth.propagator(0x51, 1, L, T, n_src, dtype=dtype)).pin_memory()
    fu, fd = hu.cuda(), hd.cuda()
    nan = float("nan")
    du = torch.full_like(fu, complex(nan, nan))
    dd = torch.full_like(fd, complex(nan, nan))
    n = wick.wick_upload_rows(hu, hd, du, dd, tabs, L, T, n_src, mode=mode)
    torch.cuda.synchronize()
    # upper-spin tables: rows (a, alpha), alpha in {0, 1}, of both flavours
    up = [0, 1, 4, 5, 8, 9]
    lo = [2, 3, 6, 7, 10, 11]
    assert n == 2 * n_src * T * L ** 3 * len(up) * 12 * hu.element_size()
    S = du.view(n_src, T, L ** 3, 12, 12).cpu()
    H = hu.view(n_src, T, L ** 3, 12, 12)
    assert torch.isnan(S[..., lo, :].real).all()                             # untouched lower rows
    assert torch.equal(S[..., up, :], H[..., up, :])
    for prec in (wick.WICK_MIXED, wick.WICK_MIXED_SIMT, wick.WICK_FP64):
        ref = blocks(fu, fd, tabs, nuc, prec, L, T, n_src)
        got = blocks(du, dd, tabs, nuc, prec, L, T, n_src)
        assert np.array_equal(got, ref), prec


def test_upload_rejects_pageable_and_mismatch():
    L, T, n_src = 2, 1, 1
    nuc = operators.nucleus("he4")
    tabs = wick.Tables(nuc)
    h = torch.from_numpy(synth.propagator(1, 0, L, T, n_src, dtype=np.complex64))   # pageable
    d = h.cuda()
    with pytest.raises(ValueError):            # the binding refuses it before the library sees it
        wick.wick_upload_rows(h, h, d, d, tabs, L, T, n_src)
    # and so does the C ABI itself, called directly
    hp_, dp_ = (wick.wick_prop(x.data_ptr(), L, T, n_src, wick.WICK_C64) for x in (h, d))
    n = ctypes.c_size_t(0)
    assert wick.load().wick_upload_rows(ctypes.byref(hp_), ctypes.byref(hp_), ctypes.byref(dp_), ctypes.byref(dp_),
                                        tabs.ops, ctypes.byref(tabs.layout), wick.WICK_UPLOAD_DMA, ctypes.byref(n),
                                        None) == wick.WICK_EINVAL
    hp = h.pin_memory()
    d128 = torch.zeros(h.shape, dtype=torch.complex128, device="cuda")
    with pytest.raises(wick.WickError):
        wick.wick_upload_rows(hp, hp, d128, d128, tabs, L, T, n_src)
    with pytest.raises(wick.WickError):
        wick.wick_upload_rows(hp, hp, d, d, tabs, L, T, n_src, mode=7)
