"""Pins of the oracle's top-fraction pieces (Sec. V.C): per-term contributions and the ranking.

* the contributions of the reduced terms add up to the correlator -- the C table sum and the
  plain Wick sum over every raw term (the definition), on He-3 and the deuteron;
* each contribution is its term's product of antisymmetric blocks, re-derived here from the
  single-product blocks of one slice by hand for a few terms;
* the ranking takes the largest magnitudes, ties to the earlier term, at least one term, all of
  them for fraction 1.
"""
import numpy as np
import pytest

from oracle import operators as ops
from oracle import oracle as O
from paper_2411_08962_gb300 import synth


def props(L, T, n_src=1, seed=11):
    return (synth.propagator(seed, 0, L, T, n_src), synth.propagator(seed, 1, L, T, n_src))


@pytest.mark.parametrize("name", ["deuteron", "he3"])
def test_contributions_add_up_to_the_correlator(name):
    nuc = ops.nucleus(name)
    Su, Sd = props(2, 3, n_src=2)
    Bh = O.blocks_single(Su, Sd, nuc)
    tab = O.dedup(nuc)
    c = O.term_contributions(nuc, Bh, tab)
    assert c.shape == (len(tab["w"]), 2 * 3)
    total = c.sum(axis=0).reshape(2, 3)
    for ref in (O.table_correlator(nuc, Bh, tab), O.raw_correlator(nuc, Bh)):
        assert np.max(np.abs(total - ref)) / np.max(np.abs(ref)) < 1e-12


def test_contribution_is_the_product_of_antisymmetric_blocks():
    nuc = ops.nucleus("deuteron")
    Su, Sd = props(2, 1)
    Bh = O.blocks_single(Su, Sd, nuc)[0, 0]
    tab = O.dedup(nuc)
    c = O.term_contributions(nuc, Bh[None], tab)[:, 0]
    nc = len(nuc["chi"])
    for u in (0, len(tab["w"]) // 2, len(tab["w"]) - 1):
        prod = complex(tab["w"][u]) * nuc["scale"]
        for bid in tab["ids"][u]:
            bid = int(bid)
            os_, i1, i2, i3 = bid // nc ** 3, (bid // nc ** 2) % nc, (bid // nc) % nc, bid % nc
            swapped = ((os_ * nc + i2) * nc + i1) * nc + i3
            prod *= Bh[bid] - Bh[swapped]
        assert abs(c[u] - prod) <= 1e-13 * abs(prod)


def test_top_terms_ranking():
    mag = np.array([0.5, 3.0, 1.0, 3.0, 0.0, 2.0])
    assert list(O.top_terms(mag, 1.0)) == [0, 1, 2, 3, 4, 5]
    assert list(O.top_terms(mag, 0.5)) == [1, 3, 5]            # 3.0, 3.0 (ties: index order), 2.0
    assert list(O.top_terms(mag, 0.2)) == [1, 3]               # ceil(1.2) = 2
    assert list(O.top_terms(mag, 1e-9)) == [1]                 # at least one term
