"""Pins of the oracle's operator layer against textbook Dirac algebra and the
paper's Table I counts (CPU only)."""
import os
from math import factorial

import numpy as np
import pytest

from oracle import operators as ops

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_counts.txt")


def test_clifford_algebra_and_hermiticity():
    g = ops.gammas()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4))
    g5 = g[4]
    assert np.allclose(g5 @ g5, np.eye(4))
    for mu in range(4):
        assert np.allclose(g5 @ g[mu], -g[mu] @ g5)


def test_charge_conjugation_properties():
    """C = gamma4 gamma2 satisfies C gamma_mu C^-1 = -gamma_mu^T and C gamma5 is
    antisymmetric (the diquark of Eq. 1000 is a scalar)."""
    g = ops.gammas()
    Cm = ops.charge_conjugation()
    Ci = np.linalg.inv(Cm)
    for mu in range(4):
        assert np.allclose(Cm @ g[mu] @ Ci, -g[mu].T)
    cg5 = ops.cg5()
    assert np.allclose(cg5, -cg5.T)
    G = ops.integer_matrix(cg5)
    # block diagonal in the Dirac basis; upper block is +-epsilon_{alpha beta}
    assert np.all(G[:2, 2:] == 0) and np.all(G[2:, :2] == 0)
    assert abs(G[0, 1]) == 1 and G[0, 1] == -G[1, 0] and G[0, 0] == 0 and G[1, 1] == 0


def test_parity_projectors():
    for s in (+1, -1):
        P = ops.parity_projector(s)
        assert np.allclose(P @ P, P)
    assert np.allclose(ops.parity_projector(1) + ops.parity_projector(-1), np.eye(4))
    # with the upper-component restriction C g5 P+ equals C g5 on the upper block
    upper = ops.integer_matrix(ops.cg5() @ ops.parity_projector(1))
    assert np.array_equal(upper[:2, :2], ops.integer_matrix(ops.cg5())[:2, :2])
    assert np.all(upper[2:, :] == 0) and np.all(upper[:, 2:] == 0)


def test_levi_civita():
    e = ops.levi_civita()
    assert e[0, 1, 2] == 1 and e[1, 0, 2] == -1 and np.count_nonzero(e) == 6
    m = np.random.default_rng(0).standard_normal((3, 3))
    assert np.isclose(np.einsum("abc,a,b,c->", e, m[0], m[1], m[2]), np.linalg.det(m))


def test_nucleon_table_sizes():
    up = ops.nucleon_table(ops.cg5(), ops.UPPER, ops.UPPER)
    full = ops.nucleon_table(ops.cg5(), ops.ALL_SPINS, ops.ALL_SPINS)
    # 6 colour permutations x (2 resp. 4) non-zero C g5 entries per nucleon spin
    assert len(up) == 2 * 6 * 2 and len(full) == 4 * 6 * 4
    assert all(abs(e[4]) == 1 for e in full)


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, A, nu, nd, nperm, nloop = line.split()
        rows.append((name, int(A), int(nu), int(nd), nperm, nloop))
    return rows


def _matches(value, printed):
    if printed.startswith("approx:"):
        m, e = printed[7:].split("e")
        return abs(value / (float(m) * 10 ** int(e)) - 1.0) < 0.5
    return value == int(printed)


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: r[0])
def test_table1_counts(row):
    name, A, nu, nd, nperm, nloop = row
    assert nu + nd == 3 * A
    assert _matches(factorial(nu) * factorial(nd), nperm)
    assert _matches(6 ** (2 * A) * 4 ** (2 * A), nloop)


@pytest.mark.parametrize("name,nu,nd,nsrc,nsink", [
    ("deuteron", 3, 3, 144, 1), ("he3", 5, 4, 3456, 2), ("he4", 6, 6, 20736, 1)])
def test_nucleus_raw_counts(name, nu, nd, nsrc, nsink):
    nuc = ops.nucleus(name)
    assert ops.quark_counts(nuc) == (nu, nd)
    assert len(nuc["src"]) == nsrc and len(nuc["sink"]) == nsink
    assert ops.n_raw_terms(nuc) == nsink * nsrc * factorial(nu) * factorial(nd)


def test_permutation_enumeration():
    perms = ops.all_permutations(4)
    assert len(perms) == 24 and perms[0] == ((0, 1, 2, 3), 1) and perms[1] == ((0, 1, 3, 2), -1)
    assert sum(s for _, s in perms) == 0
