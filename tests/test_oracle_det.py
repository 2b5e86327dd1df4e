"""Pins of the point-sink determinant oracle (Eq. 2.9; Sec. III.C; App. A).

The oracle evaluates Eq. 2.9 with determinants by their Leibniz definition.
It is pinned against things other than itself:
  * the operator term counts printed in the paper's determinant table;
  * numpy's LU determinant;
  * the plain Wick permutation sum of the plane-wave oracle: a point sink and
    a plane-wave sink coincide on a one-site lattice, and for one nucleon on
    any lattice (the plane-wave oracle is pinned in test_oracle_pins.py);
  * gauge invariance and homogeneity;
  * antisymmetrised coefficient tables (method A) = the unantisymmetrised sum;
  * the minimal sets found by comparing index lists = those found by the
    paper's randomised identity testing mod 2^61 - 1.
"""
import os

import numpy as np
import pytest

from oracle import det as DT
from oracle import operators as ops
from oracle import oracle as O
from paper_2411_08962_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "det_table_terms.txt")


def golden_counts():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, terms, nu, nd = line.split()
            out[name] = (int(terms), int(nu), int(nd))
    return out


def props(L, T, seed, n_src=1):
    return synth.propagator(seed, 0, L, T, n_src), synth.propagator(seed, 1, L, T, n_src)


@pytest.mark.parametrize("name,builder", [("2H", ops.paper_deuteron), ("3He", lambda: ops.paper_he3(0)),
                                          ("3He", lambda: ops.paper_he3(1)), ("4He", ops.paper_he4)])
def test_operator_term_counts_match_paper_table(name, builder):
    terms, nu, nd = golden_counts()[name]
    tab, fl = builder()
    assert (sum(1 for f in fl if f == ops.U), sum(1 for f in fl if f == ops.D)) == (nu, nd)
    assert len(ops.antisymmetrised(tab, nu)) == terms


def test_he3_count_fixes_projector_sign():
    """With P+- = (1 +- gamma4)/2 of this basis the 3He operator would have 744 terms, not 1026."""
    cgp = ops.cg5() @ ops.parity_projector(+1)
    cgm = ops.cg5() @ ops.parity_projector(-1)
    o3 = [(ops.U, ops.nucleon_table(cgm, ops.ALL_SPINS, ops.ALL_SPINS)),   # p- with (1 - gamma4)/2
          (ops.D, ops.nucleon_table(cgp, ops.ALL_SPINS, ops.ALL_SPINS)),   # n+ with (1 + gamma4)/2
          (ops.U, ops.nucleon_table(cgp, ops.ALL_SPINS, ops.ALL_SPINS))]   # p+
    G = ops.integer_matrix(ops.cg5())
    terms = [((0, 1, 2), (a, b, 0), int(G[a, b])) for a in range(4) for b in range(4) if G[a, b]]
    tab, fl = ops.grouped_operator(o3, terms)
    assert len(ops.antisymmetrised(tab, 5)) == 744


@pytest.mark.parametrize("nu,nd", [(1, 1), (2, 3), (4, 2), (5, 4), (6, 6)])
def test_leibniz_determinants_match_lu(nu, nd):
    rng = np.random.default_rng(nu * 10 + nd)
    Su = rng.standard_normal((1, 1, 1, 3, 4, 3, 4)) + 1j * rng.standard_normal((1, 1, 1, 3, 4, 3, 4))
    Sd = rng.standard_normal((1, 1, 1, 3, 4, 3, 4)) + 1j * rng.standard_normal((1, 1, 1, 3, 4, 3, 4))
    ru, cu = rng.choice(12, nu, replace=False), rng.choice(12, nu, replace=False)
    rd, cd = rng.choice(12, nd, replace=False), rng.choice(12, nd, replace=False)
    g = DT.point_correlator(Su, Sd, [(tuple(ru) + tuple(rd), 1)], [(tuple(cu) + tuple(cd), 1)], nu, nd)[0, 0]
    Mu, Md = Su[0, 0, 0].reshape(12, 12), Sd[0, 0, 0].reshape(12, 12)
    ref = np.linalg.det(Mu[np.ix_(ru, cu)]) * np.linalg.det(Md[np.ix_(rd, cd)])
    assert abs(g - ref) <= 1e-13 * abs(ref)


def test_point_sink_equals_plain_wick_sum_on_one_site():
    """2H: Eq. 2.9 with determinants = the raw permutation sum of Eq. 2.8 (plane-wave oracle), V = 1."""
    tab, nu, nd, scale = DT.operator("deuteron")
    Su, Sd = props(1, 3, seed=11)
    gp = DT.point_correlator(Su, Sd, tab, tab, nu, nd, scale)
    graw = O.correlator(Su, Sd, ops.paper_point_nucleus("deuteron"))
    assert np.max(np.abs(gp - graw) / np.abs(graw)) < 1e-13


def test_point_sink_equals_reduced_plane_wave_on_one_site():
    """3He: the same against the reduced plane-wave table (antisymmetric blocks carry 2^A)."""
    tab, nu, nd, scale = DT.operator("he3")
    Su, Sd = props(1, 2, seed=12)
    gp = DT.point_correlator(Su, Sd, tab, tab, nu, nd, scale)
    nuc = ops.paper_point_nucleus("he3")
    B = O.antisymmetric_blocks(O.blocks_single(Su, Sd, nuc), nuc)
    gw = O.table_correlator(nuc, B, O.dedup(nuc))
    assert np.max(np.abs(gp - gw / 2 ** 3) / np.abs(gp)) < 1e-12


def test_one_nucleon_point_sink_equals_plane_wave():
    """A = 1: the sink of one nucleon is a point; both forms agree on any lattice."""
    nuc = ops.nucleus("proton", "full")
    tab, fl = ops.grouped_operator(nuc["ops"], [((ops.PROTON,), (1,), 1)])
    Su, Sd = props(2, 2, seed=13)
    gp = DT.point_correlator(Su, Sd, tab, tab, 2, 1)
    pw = ops._cluster(nuc["ops"], [((ops.PROTON,), (1,), 1)], 1.0)
    graw = O.correlator(Su, Sd, pw)
    assert np.max(np.abs(gp - graw) / np.abs(graw)) < 1e-13


def test_point_sink_gauge_invariance():
    """S(x) -> G(x) S(x) G0^+ (colour indices) leaves the colour-singlet point sink unchanged."""
    tab, nu, nd, scale = DT.operator("deuteron")
    Su, Sd = props(2, 1, seed=14)
    rng = np.random.default_rng(5)
    V = 8
    Gx = synth.random_su3(rng, V)
    G0 = synth.random_su3(rng, 1)[0]

    def rot(S):
        return np.einsum("xab,stxbpcq,dc->stxapdq", Gx, S, G0.conj())
    g0 = DT.point_correlator(Su, Sd, tab, tab, nu, nd)
    g1 = DT.point_correlator(rot(Su), rot(Sd), tab, tab, nu, nd)
    assert np.max(np.abs(g1 - g0) / np.abs(g0)) < 1e-12


def test_point_sink_homogeneity():
    tab, nu, nd, scale = DT.operator("deuteron")
    Su, Sd = props(2, 1, seed=15)
    lam = 1.7 - 0.4j
    g0 = DT.point_correlator(Su, Sd, tab, tab, nu, nd)
    g1 = DT.point_correlator(lam * Su, lam * Sd, tab, tab, nu, nd)
    assert np.max(np.abs(g1 - lam ** 6 * g0) / np.abs(lam ** 6 * g0)) < 1e-12


def test_antisymmetrised_tables_equal_unantisymmetrised_sum():
    """Sum over every (chi, chi') of the raw tables (unsorted determinants) = method A."""
    nuc = ops.nucleus("proton", "full")
    tab, fl = ops.grouped_operator(nuc["ops"], [((ops.PROTON,), (0,), 1), ((ops.PROTON,), (3,), 2)])
    pu, pd, iu, idd, t_pu, t_pd, t_w = [], [], {}, {}, [], [], []
    for chi, w in tab:
        for chi2, w2 in tab:
            ku, kd = (chi[:2], chi2[:2]), (chi[2:], chi2[2:])
            for key, lst, idx in ((ku, pu, iu), (kd, pd, idd)):
                if key not in idx:
                    idx[key] = len(lst)
                    lst.append(key)
            t_pu.append(iu[ku])
            t_pd.append(idd[kd])
            t_w.append(w * w2)
    raw = dict(pu=pu, pd=pd, t_pu=np.array(t_pu), t_pd=np.array(t_pd), t_w=np.array(t_w))
    Su, Sd = props(2, 2, seed=16)
    g_raw = DT.point_correlator(Su, Sd, None, None, 2, 1, structure=raw)
    g_a = DT.point_correlator(Su, Sd, tab, tab, 2, 1)
    assert np.max(np.abs(g_raw - g_a) / np.abs(g_a)) < 1e-12


@pytest.mark.parametrize("name", ["deuteron", "he3"])
def test_minimal_sets_by_identity_testing(name):
    """Comparing index lists and randomised identity testing mod p give the same minimal sets."""
    tab, nu, nd, _ = DT.operator(name)
    zu, zd, th = DT.minimal_sets(tab, tab, nu)
    mu, md, mth = DT.minimal_sets_modp(tab, tab, nu, nd)
    assert mu == zu and md == zd and mth == th
    n = len(ops.antisymmetrised(tab, nu))
    assert len(th) == n * n      # no two (M, M') pairs share both determinants


def test_minimal_set_reduced_sum_equals_term_sum():
    """Eq. a1 (Theta over the minimal sets) = Eq. 2.9 term by term, exactly in integer arithmetic mod p."""
    tab, nu, nd, _ = DT.operator("deuteron")
    zu, zd, th = DT.minimal_sets(tab, tab, nu)
    st = DT.pair_structure(tab, tab, nu)
    P = DT.P61
    Mu, Md = DT.random_matrix_modp(99, 0, 0), DT.random_matrix_modp(99, 0, 1)
    du = [int(x) for x in DT.det_modp(Mu, zu, nu)]
    dd = [int(x) for x in DT.det_modp(Md, zd, nd)]
    reduced = sum(w * du[k] % P * dd[l] for (k, l), w in th.items()) % P
    terms = sum(int(w) * du[k] % P * dd[l] for k, l, w in zip(st["t_pu"], st["t_pd"], st["t_w"])) % P
    assert reduced == terms


def test_cross_pair_point_sink_equals_plain_wick_sum_on_one_site():
    """A correlation-matrix element with different sink and source operators (Eq. E3):
    n^T (C g5 P+) p at the sink, n+^T (C g5 P+) p+ at the source, against the plane-wave
    oracle's raw Wick sum with both nucleon kinds as block types, V = 1."""
    (t1, fl1), _, (t3, fl3) = ops.deuteron_basis()
    tab = ops.nucleon_table(ops.cg5() @ ops.paper_projector(+1), ops.ALL_SPINS, ops.ALL_SPINS)
    o4 = ops.plain_nucleons() + [(ops.U, tab), (ops.D, tab)]     # p, n, p+, n+
    G = ops.integer_matrix(ops.cg5() @ ops.paper_projector(+1))
    sink = sorted(((ops.NEUTRON, ops.PROTON), (a, b), int(G[a, b])) for a in range(4) for b in range(4) if G[a, b])
    nuc = dict(A=2, ops=o4, n_spin=4, chi=list(range(12)), sink=sink, src=t3, src_flav=fl3, scale=1.0)
    Su, Sd = props(1, 2, seed=17)
    gp = DT.point_correlator(Su, Sd, t1, t3, 3, 3)
    graw = O.correlator(Su, Sd, nuc)
    assert np.max(np.abs(gp - graw) / np.abs(graw)) < 1e-13


@pytest.mark.parametrize("name,flavour", [("deuteron", 0), ("deuteron", 1), ("he3", 1)])
def test_three_point_is_derivative_of_two_point(name, flavour):
    """The current through a sequential propagator Sigma_f: G3 = d/de G(S_f + e Sigma_f) at e = 0.
    G is a polynomial of degree n_f in e; its linear coefficient comes from n_f + 1 evaluations
    of the two-point oracle (exact interpolation)."""
    tab, nu, nd, scale = DT.operator(name)
    L = 2 if name == "deuteron" else 1
    Su, Sd = props(L, 1, seed=21)
    Sig = synth.propagator(22, 0, L, 1, 1)
    n_f = nu if flavour == 0 else nd
    eps = np.linspace(-1.0, 1.0, n_f + 1)
    vals = []
    for e in eps:
        a, b = (Su + e * Sig, Sd) if flavour == 0 else (Su, Sd + e * Sig)
        vals.append(DT.point_correlator(a, b, tab, tab, nu, nd, scale)[0, 0])
    coef = np.linalg.solve(np.vander(eps, n_f + 1, increasing=True).astype(complex), np.array(vals))
    g3 = DT.point_3pt(Su, Sd, Sig, flavour, tab, tab, nu, nd, scale)[0, 0]
    assert abs(g3 - coef[1]) < 1e-9 * np.max(np.abs(vals))


def test_three_point_euler_identity():
    """With Sigma_f = S_f the derivative is n_f times the two-point function (homogeneity)."""
    tab, nu, nd, scale = DT.operator("deuteron")
    Su, Sd = props(2, 2, seed=23)
    g = DT.point_correlator(Su, Sd, tab, tab, nu, nd, scale)
    assert np.max(np.abs(DT.point_3pt(Su, Sd, Su, 0, tab, tab, nu, nd, scale) - nu * g) / np.abs(g)) < 1e-13
    assert np.max(np.abs(DT.point_3pt(Su, Sd, Sd, 1, tab, tab, nu, nd, scale) - nd * g) / np.abs(g)) < 1e-13


def test_proton_three_point_point_equals_plane_wave_derivative():
    """One nucleon (the paper's proton example): the point-sink three-point function is the
    derivative of the plane-wave two-point function in the direction Sigma_u, on any lattice."""
    nuc = ops.nucleus("proton", "full")
    tab, fl = ops.grouped_operator(nuc["ops"], [((ops.PROTON,), (0,), 1), ((ops.PROTON,), (1,), 1)])
    pw = ops._cluster(nuc["ops"], [((ops.PROTON,), (0,), 1), ((ops.PROTON,), (1,), 1)], 1.0)
    Su, Sd = props(2, 1, seed=24)
    Sig = synth.propagator(25, 0, 2, 1, 1)
    eps = np.array([-1.0, 0.0, 1.0])
    vals = [O.correlator(Su + e * Sig, Sd, pw)[0, 0] for e in eps]
    coef = np.linalg.solve(np.vander(eps, 3, increasing=True).astype(complex), np.array(vals))
    g3 = DT.point_3pt(Su, Sd, Sig, 0, tab, tab, 2, 1)[0, 0]
    assert abs(g3 - coef[1]) < 1e-11 * np.max(np.abs(vals))
