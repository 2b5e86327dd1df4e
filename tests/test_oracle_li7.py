"""Pins of the oracle's Li-7 cluster operators (Sec. III.C, Eqs. He4_op, Li7).

* Storing source quarks flavour-grouped with the Grassmann sign of the
  reordering leaves the correlator unchanged (checked on He-3);
* the triton reduction equals its plain Wick sum exactly mod 2^61 - 1;
* the He-4 cluster reduction is tied to the single-product He-4 -- whose
  table is pinned to its plain sum -- through linearity in the sink and the
  source operator, exactly mod p.
"""
import numpy as np
import pytest

from oracle import operators as ops
from oracle import oracle as O
from paper_2411_08962_gb300 import synth


def props(L, T, seed=31):
    return synth.propagator(seed, 0, L, T, 1), synth.propagator(seed, 1, L, T, 1)


def test_flavour_grouped_source_is_the_same_operator():
    std = ops.nucleus("he3")
    grouped = ops._cluster(ops.nucleon_ops("upper"),
                           [((0, 0, 1), (0, 1, 0), 1), ((0, 0, 1), (1, 0, 0), -1)], 1.0)
    grouped["n_spin"], grouped["chi"] = std["n_spin"], std["chi"]
    assert grouped["src_flav"] == [0] * 5 + [1] * 4 and std["src_flav"] != grouped["src_flav"]
    Su, Sd = props(2, 1)
    assert np.allclose(O.correlator(Su, Sd, grouped), O.correlator(Su, Sd, std), rtol=1e-12, atol=0)


def test_triton_reduced_equals_plain_sum_mod_p():
    nuc = ops.triton_cluster()
    tab = O.dedup(nuc)
    assert tab["stats"][3] == len(tab["w"]) > 10 ** 6
    for seed in (5, 6):
        assert O.modp_table(nuc, tab, seed) == O.modp_raw(nuc, seed)


def _single(nuc, sink=None, src_terms=None):
    one = dict(nuc)
    if sink is not None:
        one["sink"] = [sink]
    if src_terms is not None:
        g = ops._cluster(nuc["ops"], src_terms, 1.0)
        one["src"], one["src_flav"] = g["src"], g["src_flav"]
    return one


def test_he4_cluster_by_linearity_mod_p():
    nuc = ops.he4_cluster()
    seed = 99
    full = O.modp_table(nuc, O.dedup(nuc), seed)
    p = (1 << 61) - 1
    # linearity in the sink: C(O, O) = sum_a W_a C(a, O)
    acc = 0
    for types, spins, w in nuc["sink"]:
        sub = _single(nuc, sink=(types, spins, 1))
        acc = (acc + w * O.modp_table(sub, O.dedup(sub), seed)) % p
    assert acc == full
    # linearity in the source for the first sink term: C(a, O) = sum_b W_b C(a, b)
    a = nuc["sink"][0]
    lhs_nuc = _single(nuc, sink=(a[0], a[1], 1))
    lhs = O.modp_table(lhs_nuc, O.dedup(lhs_nuc), seed)
    rhs = 0
    for types, spins, w in nuc["sink"]:
        sub = _single(nuc, sink=(a[0], a[1], 1), src_terms=[(types, spins, 1)])
        rhs = (rhs + w * O.modp_table(sub, O.dedup(sub), seed)) % p
    assert lhs == rhs


def test_he4_cluster_contains_the_single_product_he4():
    """The (p+ up, p+ down, n+ up, n+ down) x itself pair of the cluster is the
    single-product He-4 of the workloads, whose table is pinned to its plain sum."""
    nuc = ops.he4_cluster()
    term = ((ops.P_PLUS, ops.P_PLUS, ops.N_PLUS, ops.N_PLUS), (0, 1, 0, 1), 1)
    sub = _single(nuc, sink=term, src_terms=[term])
    sub["scale"] = 1.0                     # the cluster's 1/96 normalises the full operator only
    std = ops.nucleus("he4")
    Su, Sd = props(2, 1, seed=8)
    # blocks of the two layouts differ; compare correlators through the oracle's reduced sums
    c_sub = O.table_correlator(sub, O.blocks_single(Su, Sd, sub), O.dedup(sub))
    c_std = O.table_correlator(std, O.blocks_single(Su, Sd, std), O.dedup(std))
    assert np.allclose(c_sub, c_std, rtol=1e-12, atol=0)
