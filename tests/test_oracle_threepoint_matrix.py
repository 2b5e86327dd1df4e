"""Pins of the oracle's plane-wave three-point function and correlation-matrix elements.

Three-point (Sec. IV.A): the coefficient extraction is checked against
* Euler's identity for a homogeneous polynomial: with Sig = S_f the derivative in the direction
  S_f is n_f times the correlator;
* linearity in Sig;
* the proton with the current on d (one d quark, so the correlator is linear in S_d): the
  three-point function is the two-point function with S_d replaced by Sig;
* the reduced-table evaluation against the plain Wick sum.
Matrix (Eqs. E1-E3): a diagonal element is the operator's own correlator; the element of a
source and sink that differ is the plain Wick sum of that (sink, source) pair; the plane-wave
NP operator's reduced table reproduces its plain Wick sum.
"""
import numpy as np
import pytest

from oracle import operators as ops
from oracle import oracle as O
from paper_2411_08962_gb300 import synth


def props(L, T, n_src=1, seed=13):
    return (synth.propagator(seed, 0, L, T, n_src), synth.propagator(seed, 1, L, T, n_src))


def sig(L, T, n_src=1, seed=99):
    return synth.propagator(seed, 0, L, T, n_src)


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("name,flavour", [("proton", 0), ("deuteron", 0), ("deuteron", 1), ("he3", 1)])
def test_three_point_euler(name, flavour):
    nuc = ops.nucleus(name)
    Su, Sd = props(2, 2)
    nu, nd = O.ops_quark_counts(nuc)
    S_f = Su if flavour == 0 else Sd
    c3 = O.three_point_planewave(Su, Sd, S_f, flavour, nuc)
    assert rel(c3, (nu if flavour == 0 else nd) * O.correlator(Su, Sd, nuc)) < 1e-12


def test_three_point_linear_in_sig():
    nuc = ops.nucleus("deuteron")
    Su, Sd = props(2, 2)
    s1, s2 = sig(2, 2, seed=5), sig(2, 2, seed=6)
    a = O.three_point_planewave(Su, Sd, s1, 0, nuc)
    b = O.three_point_planewave(Su, Sd, s2, 0, nuc)
    c = O.three_point_planewave(Su, Sd, s1 + 2.5 * s2, 0, nuc)
    assert rel(c, a + 2.5 * b) < 1e-12


def test_three_point_single_d_line():
    nuc = ops.nucleus("proton")
    Su, Sd = props(2, 3)
    s = sig(2, 3)
    assert rel(O.three_point_planewave(Su, Sd, s, 1, nuc), O.correlator(Su, s, nuc)) < 1e-12


def test_three_point_table_equals_raw():
    nuc = ops.nucleus("he3")
    Su, Sd = props(2, 1)
    s = sig(2, 1)
    tab = O.dedup(nuc)
    assert rel(O.three_point_planewave(Su, Sd, s, 0, nuc, tab), O.three_point_planewave(Su, Sd, s, 0, nuc)) < 1e-12


def test_matrix_elements():
    basis = ops.deuteron_pw_basis()
    Su, Sd = props(2, 2)
    for i, a in enumerate(basis):
        assert rel(O.correlator(Su, Sd, O.matrix_element(a, a)), O.correlator(Su, Sd, a)) < 1e-15
    el = O.matrix_element(basis[0], basis[1])
    assert el["sink"] == basis[0]["sink"] and el["src"] == basis[1]["src"]
    c01 = O.correlator(Su, Sd, el)
    assert np.all(np.abs(c01) > 0)
    # the third operator is the sum of the first two: its elements are the sums of theirs (linearity)
    for i in range(3):
        c = [O.correlator(Su, Sd, O.matrix_element(basis[i], basis[j])) for j in range(3)]
        assert rel(c[2], c[0] + c[1]) < 1e-12
    # the reduced table of the pair reproduces its plain Wick sum
    Bh = O.blocks_single(Su, Sd, el)
    assert rel(O.table_correlator(el, Bh, O.dedup(el)), O.raw_correlator(el, Bh)) < 1e-12


def test_np_planewave_operator():
    nuc = ops.deuteron_np_planewave()
    assert nuc["A"] == 2 and nuc["n_spin"] == 4 and len(nuc["chi"]) == 12
    assert len(nuc["sink"]) == 2                      # C gamma5 P+ keeps one 2 x 2 block: two entries
    Su, Sd = props(2, 1)
    Bh = O.blocks_single(Su, Sd, nuc)
    assert rel(O.table_correlator(nuc, Bh, O.dedup(nuc)), O.raw_correlator(nuc, Bh)) < 1e-12
