"""Pins of the CPU reference against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: the printed
single-proton expression (App. B), the printed block of Eq. 2.4, a quark-level
Wick contraction on a tiny lattice, SU(3) gauge invariance, homogeneity in each
flavour, isospin symmetry, the fermion sign of reordering nucleons, and exact
modular identities of the reduced tables (Theorem 1, App. C).
"""
from itertools import product
from math import factorial

import numpy as np
import pytest

from oracle import operators as ops
from oracle import oracle as O
from paper_2411_08962_gb300 import synth


def props(L, T, n_src=1, seed=7):
    return (synth.propagator(seed, 0, L, T, n_src), synth.propagator(seed, 1, L, T, n_src))


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def custom_nucleus(ops_list, n_spin, types, sink_spins, src_spins):
    """One sink spin tuple and one source spin tuple (weights 1)."""
    return dict(A=len(types), ops=ops_list, n_spin=n_spin,
                chi=[c for c in range(12) if (c % 4) < n_spin],
                sink=[(tuple(types), tuple(sink_spins), 1)],
                src=ops.source_terms(ops_list, types, [(tuple(src_spins), 1)]),
                src_flav=ops.source_flavours(ops_list, types), scale=1.0)


# --------------------------------------------------------------------------
# App. B: the single-proton two-term expression, any spin matrix Gamma
# --------------------------------------------------------------------------
@pytest.mark.parametrize("same_flavour", [True, False])
def test_proton_closed_form(same_flavour):
    rng = np.random.default_rng(3)
    G = rng.integers(-2, 3, size=(4, 4))            # any integer diquark matrix
    tab = ops.nucleon_table(G.astype(complex), ops.ALL_SPINS, ops.ALL_SPINS)
    ops_list = [(ops.U, tab), (ops.D, tab)]
    Su, Sd = props(2, 2)
    if same_flavour:
        Sd = Su
    eps = np.zeros((3, 3, 3))
    for (a, b, c), s in (((0, 1, 2), 1), ((1, 2, 0), 1), ((2, 0, 1), 1),
                         ((1, 0, 2), -1), ((0, 2, 1), -1), ((2, 1, 0), -1)):
        eps[a, b, c] = s
    for al in range(4):
        for alp in range(4):
            nuc = custom_nucleus(ops_list, 4, (0,), (al,), (alp,))
            C = O.correlator(Su, Sd, nuc)
            # + eps_ijk G_bg eps_i'j'k' G_b'g' S_(i al, i' al') S_(j b, j' b') S_(k g, k' g')
            # - eps_ijk G_bg eps_i'j'k' G_b'g' S_(i al, j' b') S_(j b, i' al') S_(k g, k' g')
            u = Su.reshape(Su.shape[:3] + (3, 4, 3, 4))
            d = Sd.reshape(Sd.shape[:3] + (3, 4, 3, 4))
            direct = np.einsum("ijk,bg,IJK,BH,stxiI,stxjbJB,stxkgKH->st",
                               eps, G, eps, G, u[..., :, al, :, alp], u, d)
            exch = np.einsum("ijk,bg,IJK,BH,stxiJB,stxjbI,stxkgKH->st",
                             eps, G, eps, G, u[..., :, al, :, :], u[..., :, :, :, alp], d)
            ref = direct - exch
            assert rel(C, ref) < 1e-13, (al, alp)


# --------------------------------------------------------------------------
# Eq. 2.4 as printed: sink-side exchange (a<->b, alpha<->beta)
# --------------------------------------------------------------------------
def test_block_matches_eq_2_4():
    Su, Sd = props(2, 1)
    nuc = ops.nucleus("deuteron", form="full")
    B = O.antisymmetric_blocks(O.blocks_single(Su, Sd, nuc), nuc)
    B = B.reshape(1, 1, 2, 4, 12, 12, 12)
    G = ops.integer_matrix(ops.cg5())
    e = ops.levi_civita()
    for f1, f2, o in ((Su, Sd, 0), (Sd, Su, 1)):
        q1 = f1[0, 0].reshape(-1, 3, 4, 12)
        q2 = f2[0, 0].reshape(-1, 3, 4, 12)
        for al in range(4):
            direct = np.einsum("abc,mn,xaP,xbmQ,xcnR->PQR", e, G, q1[:, :, al, :], q1, q2)
            swap = np.einsum("abc,mn,xbmP,xaQ,xcnR->PQR", e, G, q1, q1[:, :, al, :], q2)
            assert rel(B[0, 0, o, al], direct - swap) < 1e-13


# --------------------------------------------------------------------------
# quark-level Wick contraction on a 2^3 lattice (no blocks)
# --------------------------------------------------------------------------
def test_deuteron_quark_level_brute_force():
    nuc = ops.nucleus("deuteron")
    L, V = 2, 8
    Su, Sd = props(L, 1)
    S = [Su[0, 0].reshape(V, 12, 12), Sd[0, 0].reshape(V, 12, 12)]
    tabs = [[e for e in nuc["ops"][o][1] if e[0] == 0] for o in (0, 1)]
    sink = [(ep, en) for ep in tabs[0] for en in tabs[1]]               # p(up) n(up)
    sink_chi = np.array([e1[1:4] + e2[1:4] for e1, e2 in sink])        # (144, 6)
    sink_w = np.array([e1[4] * e2[4] for e1, e2 in sink])
    src_chi = np.array([c for c, _ in nuc["src"]])                      # (144, 6)
    src_w = np.array([w for _, w in nuc["src"]])
    flav = [0, 0, 1, 1, 1, 0]
    upos = [q for q in range(6) if flav[q] == 0]
    dpos = [q for q in range(6) if flav[q] == 1]
    total = 0.0
    for (pu, _), (pd, _) in product(ops.all_permutations(3), ops.all_permutations(3)):
        # sink quark q is paired with source position pos[q]; the Grassmann sign
        # is the parity of that pairing as a permutation of the six quarks
        pos = [0] * 6
        for m, q in enumerate(upos):
            pos[q] = upos[pu[m]]
        for m, q in enumerate(dpos):
            pos[q] = dpos[pd[m]]
        inv = sum(1 for a in range(6) for b in range(a + 1, 6) if pos[a] > pos[b])
        sgn = -1 if inv % 2 else 1
        for x1 in range(V):
            for x2 in range(V):
                prod_ = np.ones((len(sink), len(src_w)), dtype=complex)
                for q in range(6):
                    x = x1 if q < 3 else x2
                    prod_ *= S[flav[q]][x][sink_chi[:, q][:, None], src_chi[:, pos[q]][None, :]]
                total += sgn * np.sum(sink_w[:, None] * src_w[None, :] * prod_)
    C = O.correlator(Su, Sd, nuc)
    assert abs(C[0, 0] - total) / abs(total) < 1e-12


# --------------------------------------------------------------------------
# symmetries
# --------------------------------------------------------------------------
def gauge_transform(S, Gx, G0):
    """S(x) -> G(x) S(x) G0^dagger on the colour indices."""
    s = S.reshape(S.shape[:3] + (3, 4, 3, 4))
    out = np.einsum("xab,stxbuce,dc->stxaude", Gx, s, G0.conj())
    return out.reshape(S.shape)


@pytest.mark.parametrize("name", ["deuteron", "he3"])
def test_su3_gauge_invariance(name):
    nuc = ops.nucleus(name)
    L, T = 2, 1
    Su, Sd = props(L, T)
    rng = np.random.default_rng(11)
    Gx = synth.random_su3(rng, L ** 3)
    G0 = synth.random_su3(rng, 1)[0]
    C0 = O.correlator(Su, Sd, nuc)
    C1 = O.correlator(gauge_transform(Su, Gx, G0), gauge_transform(Sd, Gx, G0), nuc)
    assert rel(C1, C0) < 1e-12


def test_blocks_sink_gauge_invariant():
    nuc = ops.nucleus("deuteron", form="full")
    Su, Sd = props(2, 1)
    Gx = synth.random_su3(np.random.default_rng(5), 8)
    one = np.eye(3)
    B0 = O.blocks_single(Su, Sd, nuc)
    B1 = O.blocks_single(gauge_transform(Su, Gx, one), gauge_transform(Sd, Gx, one), nuc)
    assert rel(B1, B0) < 1e-12


@pytest.mark.parametrize("name", ["deuteron", "he3"])
def test_homogeneity_per_flavour(name):
    nuc = ops.nucleus(name)
    nu, nd = ops.quark_counts(nuc)
    Su, Sd = props(2, 1)
    lu, ld = 0.7 + 0.3j, -1.1 + 0.2j
    C0 = O.correlator(Su, Sd, nuc)
    C1 = O.correlator(lu * Su, ld * Sd, nuc)
    assert rel(C1, lu ** nu * ld ** nd * C0) < 1e-12


def test_isospin_blocks():
    nuc = ops.nucleus("deuteron", form="full")
    Su, _ = props(2, 1)
    B = O.blocks_single(Su, Su, nuc).reshape(1, 1, 2, -1)
    assert np.array_equal(B[:, :, 0], B[:, :, 1])


@pytest.mark.parametrize("name,order,sign", [
    ("deuteron", (1, 0), -1),        # p n -> n p : 3 x 3 quark transpositions
    ("he3", (0, 2, 1), -1),          # p p n -> p n p
    ("he3", (2, 0, 1), +1),          # p p n -> n p p : n moves past 6 quarks
])
def test_fermion_sign_of_nucleon_reordering(name, order, sign):
    """Reordering the source nucleon operators (Grassmann-odd) multiplies the
    correlator by the parity of the induced quark permutation."""
    nuc = ops.nucleus(name)
    A = nuc["A"]
    types = [t for t in nuc["sink"][0][0]]
    new_src = {}
    for chi, w in nuc["src"]:
        groups = [chi[3 * k:3 * k + 3] for k in range(A)]
        new = tuple(x for k in order for x in groups[k])
        new_src[new] = new_src.get(new, 0) + w
    re = dict(nuc)
    re["src"] = sorted(new_src.items())
    re["src_flav"] = ops.source_flavours(nuc["ops"], [types[k] for k in order])
    Su, Sd = props(2, 1)
    C0 = O.correlator(Su, Sd, nuc)
    C1 = O.correlator(Su, Sd, re)
    assert rel(C1, sign * C0) < 1e-12


# --------------------------------------------------------------------------
# the reduced tables (Sec. III.B, App. C)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["proton", "deuteron", "he3"])
def test_reduced_equals_raw_fp64(name):
    nuc = ops.nucleus(name)
    Su, Sd = props(2, 2, n_src=2)
    Bh = O.blocks_single(Su, Sd, nuc)
    tab = O.dedup(nuc)
    assert rel(O.table_correlator(nuc, Bh, tab), O.raw_correlator(nuc, Bh)) < 1e-12
    ms = O.source_multisets(nuc)
    nu, nd = ops.quark_counts(nuc)
    assert tab["stats"][0] == ms["n_red"] == len(nuc["sink"]) * len(ms["CM"]) * factorial(nu) * factorial(nd)


@pytest.mark.parametrize("name", ["deuteron", "he3"])
def test_reduced_equals_raw_mod_p(name):
    """Exact identity at fresh random integer points, independent of the
    points used to build the table."""
    nuc = ops.nucleus(name)
    tab = O.dedup(nuc, seed=1)
    for seed in (101, 202, 303):
        assert O.modp_table(nuc, tab, seed) == O.modp_raw(nuc, seed)


def test_modp_detects_a_dropped_term():
    nuc = ops.nucleus("deuteron")
    tab = O.dedup(nuc)
    bad = dict(ids=tab["ids"][1:], w=tab["w"][1:])
    assert O.modp_table(nuc, bad, 77) != O.modp_raw(nuc, 77)


@pytest.mark.parametrize("name", ["deuteron", "he3"])
def test_hash_partition_equals_symbolic(name):
    nuc = ops.nucleus(name)
    a = O.dedup(nuc, mode="hash")
    b = O.dedup(nuc, mode="symbolic")
    for k in ("rep", "w", "ids"):
        assert np.array_equal(a[k], b[k])
    assert a["stats"] == b["stats"]


def test_table_independent_of_seed_and_sites():
    """The minimal set depends on the operator only (Sec. III.B)."""
    nuc = ops.nucleus("he3")
    ref = O.dedup(nuc, seed=1, V0=1)
    for seed, V0 in ((2, 1), (3, 2), (99, 3)):
        t = O.dedup(nuc, seed=seed, V0=V0)
        for k in ("rep", "w", "ids"):
            assert np.array_equal(t[k], ref[k])


def test_deuteron_at_most_nine_classes_per_source_tuple():
    """n_u! n_d! / 2^A = 9 independent terms for a fixed source tuple (Sec. IV)."""
    nuc = ops.nucleus("deuteron")
    counts = []
    for chi, w in nuc["src"]:
        one = dict(nuc)
        one["src"] = [(chi, w)]
        t = O.dedup(one)
        counts.append(len(t["w"]))
        # one source tuple: one multiset (3! 3! orderings) unless a flavour repeats an index
        assert t["stats"][0] in (0, factorial(3) * factorial(3))
    assert max(counts) <= 9 and max(counts) > 0


def test_antisymmetrised_source():
    """Method B of Sec. III.C: the source collapses onto sorted multisets.  For
    He-4 (6 u and 6 d quarks in 6 upper colour-spin states each) Pauli leaves
    exactly one multiset pair, every state once; its weight is the signed sum
    of all 12^4 product tuples that are reorderings of it."""
    he4 = O.source_multisets(ops.nucleus("he4"))
    assert len(he4["CM"]) == 1 and he4["n_red"] == factorial(6) ** 2
    assert list(he4["Mu"][0]) == list(range(6)) and list(he4["Md"][0]) == list(range(6))
    # brute force over the source tuples for the weight
    nuc = ops.nucleus("he4")
    flav = nuc["src_flav"]
    tot = 0
    for chi, w in nuc["src"]:
        u = [c for c, f in zip(chi, flav) if f == 0]
        d = [c for c, f in zip(chi, flav) if f == 1]
        if len(set(u)) == 6 and len(set(d)) == 6:
            inv = sum(a > b for seq in (u, d) for i, a in enumerate(seq) for b in seq[i + 1:])
            tot += w * (-1) ** inv
    assert he4["CM"][0] == tot and tot != 0


def test_weights_are_integers_after_pair_folding():
    for name in ("deuteron", "he3"):
        t = O.dedup(ops.nucleus(name))
        assert t["w"].dtype == np.int64 and np.all(t["w"] != 0)
        assert np.all(np.diff(t["rep"]) > 0)
